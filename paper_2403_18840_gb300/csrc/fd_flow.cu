// Affine coupling normalizing flow on the unit hypercube (Appendix A:
// composition of coupling layers, Eq. coupling_layer; density by change of
// variables, Eq. NFtransform; forward-KL training).  Hand-written BF16
// tensor-core kernels (mma.sync m16n8k16, FP32 accumulation) for sm_103a.
//
// Layer l: the conditioning half A (first ceil(D/2) coordinates on even
// layers, the rest on odd ones) feeds an MLP a -> 128 -> 128 -> 2b (ReLU);
// its outputs are s_raw (rows 0..b-1 of W3) and t (rows b..2b-1);
// s = 5 tanh(s_raw / 5); y_B <- y_B exp(s) + t.  The flow acts in logit space:
// y = logit(z) for the uniform base z, x = sigmoid(y).
//
// Device layout of one layer's BF16 weights (contiguous, 16-byte aligned,
// staged into shared memory by one 1-D TMA bulk copy):
//   W1p [128][24]  (in padded 16, row stride 24)      6144 B
//   W2  [128][136] (row stride 136)                  34816 B
//   W3p [32][136]  (rows 0..15 s_raw, 16..31 t)       8704 B
//   b1 [128], b2 [128], b3p [32] FP32                  1152 B
// Warp tiles are 16 samples; the three GEMMs chain in registers (accumulator
// fragments become the next GEMM's A fragments).
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "fd_internal.cuh"

namespace {

constexpr int H = 128;
constexpr int W1_LD = 24, W2_LD = 136, W3_LD = 136;
constexpr int OFF_W1 = 0;
constexpr int OFF_W2 = OFF_W1 + H * W1_LD * 2;        // 6144
constexpr int OFF_W3 = OFF_W2 + H * W2_LD * 2;        // 40960
constexpr int OFF_B1 = OFF_W3 + 32 * W3_LD * 2;       // 49664
constexpr int OFF_B2 = OFF_B1 + H * 4;
constexpr int OFF_B3 = OFF_B2 + H * 4;
constexpr int LAYER_BYTES = OFF_B3 + 32 * 4;          // 50816
constexpr int YS = 24;                                // padded coordinates per sample row
constexpr float S_CLAMP = 5.0f;
constexpr uint32_t WAIT_LIMIT = 1u << 24;

static_assert(LAYER_BYTES % 16 == 0, "layer block must be 16-byte sized");

struct FlowDims {
    int D, K, h;          // dimension, layers, first-half size ceil(D/2)
};

__device__ __forceinline__ int a_size(const FlowDims &f, int l) { return (l % 2 == 0) ? f.h : f.D - f.h; }
__device__ __forceinline__ int b_size(const FlowDims &f, int l) { return (l % 2 == 0) ? f.D - f.h : f.h; }
__device__ __forceinline__ int a_idx(const FlowDims &f, int l, int i) { return (l % 2 == 0) ? i : f.h + i; }
__device__ __forceinline__ int b_idx(const FlowDims &f, int l, int j) { return (l % 2 == 0) ? f.h + j : j; }

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&v);
}
__device__ __forceinline__ float bf_lo(uint32_t v) { return __uint_as_float(v << 16); }
__device__ __forceinline__ float bf_hi(uint32_t v) { return __uint_as_float(v & 0xFFFF0000u); }

__device__ __forceinline__ void mma16816(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// B fragment of B[k][n] = W[n][k] (W row-major [n][k], i.e. B column-major)
__device__ __forceinline__ void bfrag(const __nv_bfloat16 *W, int ld, int kt, int nt, int g, int t, uint32_t &b0,
                                      uint32_t &b1) {
    const __nv_bfloat16 *p = W + (nt * 8 + g) * ld + kt * 16 + 2 * t;
    b0 = *reinterpret_cast<const uint32_t *>(p);
    b1 = *reinterpret_cast<const uint32_t *>(p + 8);
}
// B fragments of n-tiles nt0 and nt0 + 1 at k-step kt with one ldmatrix.x4
// (W row-major [n][k], rows 16-byte aligned): lanes 8m..8m+7 address row r of
// 8x8 matrix m = (n-tile nt0 + m/2, k half m%2); b[0..1] belong to nt0, b[2..3]
// to nt0 + 1, in the register order of the m16n8k16 B operand.
__device__ __forceinline__ void bfrag2(const __nv_bfloat16 *W, int ld, int kt, int nt0, int lane, uint32_t (&b)[4]) {
    const int m = lane >> 3, r = lane & 7;
    const __nv_bfloat16 *p = W + ((nt0 + (m >> 1)) * 8 + r) * ld + kt * 16 + (m & 1) * 8;
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(b[0]), "=r"(b[1]), "=r"(b[2]), "=r"(b[3])
                 : "r"((uint32_t)__cvta_generic_to_shared(p)));
}
// B fragment of B[k][n] = W[k][n] (W row-major [k][n]: transposed access)
__device__ __forceinline__ void bfrag_t(const __nv_bfloat16 *W, int ld, int kt, int nt, int g, int t, uint32_t &b0,
                                        uint32_t &b1) {
    const uint16_t *p = reinterpret_cast<const uint16_t *>(W) + (kt * 16 + 2 * t) * ld + nt * 8 + g;
    b0 = (uint32_t)p[0] | ((uint32_t)p[ld] << 16);
    b1 = (uint32_t)p[8 * ld] | ((uint32_t)p[9 * ld] << 16);
}

// accumulator tiles (2j, 2j+1) -> A fragment of k-tile j
// ReLU and round two FP32 values to a packed BF16 pair (lo in the low half)
__device__ __forceinline__ uint32_t relu_pack(float lo, float hi) {
    uint32_t d;
    asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    return d;
}
// accumulators of n-tiles (2j, 2j+1) -> A fragment of the next layer, with ReLU
__device__ __forceinline__ void c_to_a_relu(const float (&c0)[4], const float (&c1)[4], uint32_t (&a)[4]) {
    a[0] = relu_pack(c0[0], c0[1]);
    a[1] = relu_pack(c0[2], c0[3]);
    a[2] = relu_pack(c1[0], c1[1]);
    a[3] = relu_pack(c1[2], c1[3]);
}
__device__ __forceinline__ void c_to_a(const float (&c0)[4], const float (&c1)[4], uint32_t (&a)[4]) {
    a[0] = pack_bf16(c0[0], c0[1]);
    a[1] = pack_bf16(c0[2], c0[3]);
    a[2] = pack_bf16(c1[0], c1[1]);
    a[3] = pack_bf16(c1[2], c1[3]);
}

struct LayerSmem {
    const __nv_bfloat16 *W1, *W2, *W3;
    const float *b1, *b2, *b3;
};

__device__ __forceinline__ LayerSmem layer_view(const unsigned char *base) {
    LayerSmem L;
    L.W1 = reinterpret_cast<const __nv_bfloat16 *>(base + OFF_W1);
    L.W2 = reinterpret_cast<const __nv_bfloat16 *>(base + OFF_W2);
    L.W3 = reinterpret_cast<const __nv_bfloat16 *>(base + OFF_W3);
    L.b1 = reinterpret_cast<const float *>(base + OFF_B1);
    L.b2 = reinterpret_cast<const float *>(base + OFF_B2);
    L.b3 = reinterpret_cast<const float *>(base + OFF_B3);
    return L;
}

// MLP on one 16-sample tile: input A fragment (16 x 16, zero-padded) ->
// h1, h2 as A fragments (post-ReLU, BF16) and o = [s_raw | t] accumulators.
// Forward MLP of one 16-row tile: accumulators start at the bias (the MMA adds
// the products to it), ReLU and the BF16 rounding of the next layer's A
// fragment are one cvt per pair.
__device__ __forceinline__ void mlp_forward(const LayerSmem &L, const uint32_t (&ain)[4], uint32_t (&h1a)[8][4],
                                            uint32_t (&h2a)[8][4], float (&o)[4][4], int g, int t) {
    const int lane = g * 4 + t;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const float u0 = L.b1[16 * j + 2 * t], u1 = L.b1[16 * j + 2 * t + 1];
        const float u2 = L.b1[16 * j + 8 + 2 * t], u3 = L.b1[16 * j + 9 + 2 * t];
        float c0[4] = {u0, u1, u0, u1}, c1[4] = {u2, u3, u2, u3};
        uint32_t b[4];
        bfrag2(L.W1, W1_LD, 0, 2 * j, lane, b);
        mma16816(c0, ain, b[0], b[1]);
        mma16816(c1, ain, b[2], b[3]);
        c_to_a_relu(c0, c1, h1a[j]);
    }
    // second layer: k-steps outer, all 16 n-tiles accumulated side by side
    // (16 independent MMA chains in flight per warp)
    float c[16][4];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const float u0 = L.b2[16 * j + 2 * t], u1 = L.b2[16 * j + 2 * t + 1];
        const float u2 = L.b2[16 * j + 8 + 2 * t], u3 = L.b2[16 * j + 9 + 2 * t];
        c[2 * j][0] = u0;
        c[2 * j][1] = u1;
        c[2 * j][2] = u0;
        c[2 * j][3] = u1;
        c[2 * j + 1][0] = u2;
        c[2 * j + 1][1] = u3;
        c[2 * j + 1][2] = u2;
        c[2 * j + 1][3] = u3;
    }
#pragma unroll
    for (int kt = 0; kt < 8; ++kt) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            uint32_t b[4];
            bfrag2(L.W2, W2_LD, kt, 2 * j, lane, b);
            mma16816(c[2 * j], h1a[kt], b[0], b[1]);
            mma16816(c[2 * j + 1], h1a[kt], b[2], b[3]);
        }
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) c_to_a_relu(c[2 * j], c[2 * j + 1], h2a[j]);
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
        const float u0 = L.b3[nt * 8 + 2 * t], u1 = L.b3[nt * 8 + 2 * t + 1];
        o[nt][0] = u0;
        o[nt][1] = u1;
        o[nt][2] = u0;
        o[nt][3] = u1;
    }
#pragma unroll
    for (int kt = 0; kt < 8; ++kt) {
        uint32_t b[4];
        bfrag2(L.W3, W3_LD, kt, 0, lane, b);
        mma16816(o[0], h2a[kt], b[0], b[1]);
        mma16816(o[1], h2a[kt], b[2], b[3]);
        bfrag2(L.W3, W3_LD, kt, 2, lane, b);
        mma16816(o[2], h2a[kt], b[0], b[1]);
        mma16816(o[3], h2a[kt], b[2], b[3]);
    }
}

// A fragment of the conditioning half of a 16-row tile of coordinates (smem rows of YS floats)
__device__ __forceinline__ void input_frag(const float *ys, const FlowDims &f, int l, int g, int t, uint32_t (&a)[4]) {
    const int na = a_size(f, l);
    auto v = [&](int row, int i) { return i < na ? ys[row * YS + a_idx(f, l, i)] : 0.f; };
    a[0] = pack_bf16(v(g, 2 * t), v(g, 2 * t + 1));
    a[1] = pack_bf16(v(g + 8, 2 * t), v(g + 8, 2 * t + 1));
    a[2] = pack_bf16(v(g, 8 + 2 * t), v(g, 9 + 2 * t));
    a[3] = pack_bf16(v(g + 8, 8 + 2 * t), v(g + 8, 9 + 2 * t));
}

// (row, j) of accumulator element q of n-tile nt (0..1 -> s, 2..3 -> t)
__device__ __forceinline__ int c_row(int q, int g) { return (q < 2) ? g : g + 8; }
__device__ __forceinline__ int c_col(int nt, int q, int t) { return (nt & 1) * 8 + 2 * t + (q & 1); }

// Apply the affine coupling to a 16-row tile; dir = +1 forward, -1 inverse.
// ld[row] += sum_j s (forward) / -= (inverse), reduced over the quad.
__device__ __forceinline__ void coupling(float *ys, float *ld, const FlowDims &f, int l, const float (&o)[4][4],
                                         int g, int t, float dir) {
    const int nb = b_size(f, l);
    float part[2] = {0.f, 0.f};
#pragma unroll
    for (int half = 0; half < 2; ++half) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int j = c_col(half, q, t);
            if (j < nb) {
                const int row = c_row(q, g);
                const float s = S_CLAMP * tanhf(o[half][q] * (1.0f / S_CLAMP));
                const float tt = o[half + 2][q];
                float &y = ys[row * YS + b_idx(f, l, j)];
                y = dir > 0.f ? fmaf(y, __expf(s), tt) : (y - tt) * __expf(-s);
                part[q >> 1] += s;
            }
        }
    }
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        part[r] += __shfl_xor_sync(0xffffffffu, part[r], 1);
        part[r] += __shfl_xor_sync(0xffffffffu, part[r], 2);
    }
    if (t == 0) {
        ld[g] += dir * part[0];
        ld[g + 8] += dir * part[1];
    }
}

// Points on the faces of the cube (FP32 rounds narrow edge bins and
// saturated sigmoids to exactly 0 or 1) are moved inside by one ulp before
// the logit of the inverse direction.
__device__ __forceinline__ float clamp_unit(float x) { return fminf(fmaxf(x, 1.1920929e-07f), 0.99999988f); }

__device__ __forceinline__ float log_sig_deriv(float y) {
    // log(sigmoid(y) (1 - sigmoid(y))) = -|y| - 2 log(1 + exp(-|y|))
    const float a = fabsf(y);
    return -a - 2.0f * log1pf(__expf(-a));
}

// Stage layer l's weights into smem with a TMA bulk copy; bounded wait.
__device__ __forceinline__ bool stage_layer(unsigned char *wsm, const unsigned char *wglob, int l, uint64_t *bar,
                                            uint32_t &phase) {
    __syncthreads();
    if (threadIdx.x == 0) {
        fence_proxy_async_smem();
        mbar_expect_tx(bar, LAYER_BYTES);
        bulk_g2s(wsm, wglob + (size_t)l * LAYER_BYTES, LAYER_BYTES, bar);
    }
    const bool ok = mbar_wait_bounded(bar, phase & 1u, WAIT_LIMIT);
    const bool anyfail = __syncthreads_or(!ok);
    if (!anyfail) ++phase;
    return !anyfail;
}

// ---- sampling / density kernel -------------------------------------------------------
// mode 0: z from Philox -> x, w = 1/q.   mode 1: x given -> log q(x).
// CTA = 4 warps; block of 64 * ROUNDS samples processed layer-major so each
// layer's weights are staged once per block.
constexpr int ROUNDS = 4;
constexpr int BLOCK = 64 * ROUNDS;

// Defensive mixture (mode 0 with n_flow < n): samples [0, n_flow) come from the
// flow, samples [n_flow, n) are uniform on the hypercube and take the inverse
// (density) pass; every sample gets w = 1 / ((1 - alpha) q(x) + alpha) with
// alpha = (n - n_flow) / n, the deterministic-mixture weight.  n_flow is a
// multiple of BLOCK (or n), so every block is of one kind.
__global__ void __launch_bounds__(128) flow_pass_kernel(const unsigned char *__restrict__ wglob, FlowDims f, int mode,
                                                         int64_t n, uint32_t seed_lo, uint32_t seed_hi,
                                                         uint32_t iter, uint32_t inst, const float *__restrict__ xin,
                                                         float *__restrict__ xout, float *__restrict__ wout,
                                                         int *status, int64_t n_flow, float alpha) {
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char *wsm = smem;
    float *ys = reinterpret_cast<float *>(smem + LAYER_BYTES);     // [BLOCK][YS]
    float *ld = ys + BLOCK * YS;                                    // [BLOCK]
    uint64_t *bar = reinterpret_cast<uint64_t *>(ld + BLOCK);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, t = lane & 3;
    if (tid == 0) {
        mbar_init(bar, 1);
        fence_mbarrier_init();
    }
    __syncthreads();
    uint32_t phase = 0;
    const int64_t nblocks = (n + BLOCK - 1) / BLOCK;
    for (int64_t blk = blockIdx.x; blk < nblocks; blk += gridDim.x) {
        const int64_t base = blk * BLOCK;
        const bool dens = mode == 1 || base >= n_flow;   // inverse (density) pass for this block
        // load / generate the block's coordinates (y = logit) and the log-Jacobian start
        for (int r = tid; r < BLOCK; r += blockDim.x) {
            const int64_t i = base + r;
            const bool valid = i < n;
            float acc = 0.f;
            if (mode == 0 && dens) {
                // defensive share: uniform x, kept as the sample, density follows
                const int64_t ii = valid ? i : base;
                const uint32_t c0 = (uint32_t)(uint64_t)ii, c1 = (uint32_t)((uint64_t)ii >> 32);
                for (int blk4 = 0; 4 * blk4 < f.D; ++blk4) {
                    const u32x4 rr = philox4x32_10(u32x4{c0, c1, iter, (inst << 8) | (uint32_t)blk4}, seed_lo, seed_hi);
                    const uint32_t wv[4] = {rr.x, rr.y, rr.z, rr.w};
                    for (int q = 0; q < 4 && 4 * blk4 + q < f.D; ++q) {
                        const float x = word_to_uniform(wv[q]);
                        const float y = __logf(x) - log1pf(-x);
                        ys[r * YS + 4 * blk4 + q] = y;
                        acc -= log_sig_deriv(y);
                        if (valid) xout[(int64_t)(4 * blk4 + q) * n + i] = x;
                    }
                }
            } else if (mode == 0) {
                const int64_t ii = valid ? i : base;
                const uint32_t c0 = (uint32_t)(uint64_t)ii, c1 = (uint32_t)((uint64_t)ii >> 32);
                for (int blk4 = 0; 4 * blk4 < f.D; ++blk4) {
                    const u32x4 rr = philox4x32_10(u32x4{c0, c1, iter, (inst << 8) | (uint32_t)blk4}, seed_lo, seed_hi);
                    const uint32_t wv[4] = {rr.x, rr.y, rr.z, rr.w};
                    for (int q = 0; q < 4 && 4 * blk4 + q < f.D; ++q) {
                        const float z = word_to_uniform(wv[q]);
                        const float y = __logf(z) - log1pf(-z);
                        ys[r * YS + 4 * blk4 + q] = y;
                        acc -= log_sig_deriv(y);            // log dy/dz
                    }
                }
            } else {
                for (int d = 0; d < f.D; ++d) {
                    const float x = clamp_unit(valid ? xin[(int64_t)d * n + i] : 0.5f);
                    const float y = __logf(x) - log1pf(-x);
                    ys[r * YS + d] = y;
                    acc -= log_sig_deriv(y);                // log q gains -log dx/dy
                }
            }
            for (int d = f.D; d < YS; ++d) ys[r * YS + d] = 0.f;
            ld[r] = acc;
        }
        for (int step = 0; step < f.K; ++step) {
            const int l = !dens ? step : f.K - 1 - step;
            if (!stage_layer(wsm, wglob, l, bar, phase)) {
                if (tid == 0 && status) atomicExch(status, DEV_ST_TIMEOUT);
                return;
            }
            const LayerSmem L = layer_view(wsm);
            for (int r = 0; r < ROUNDS; ++r) {
                float *tile = ys + (size_t)(r * 64 + warp * 16) * YS;
                float *tld = ld + r * 64 + warp * 16;
                uint32_t ain[4], h1a[8][4], h2a[8][4];
                float o[4][4];
                input_frag(tile, f, l, g, t, ain);
                mlp_forward(L, ain, h1a, h2a, o, g, t);
                coupling(tile, tld, f, l, o, g, t, !dens ? 1.f : -1.f);
                __syncwarp();
            }
        }
        __syncthreads();
        for (int r = tid; r < BLOCK; r += blockDim.x) {
            const int64_t i = base + r;
            if (i >= n) continue;
            float acc = ld[r];
            for (int d = 0; d < f.D; ++d) {
                const float y = ys[r * YS + d];
                acc += log_sig_deriv(y);
                if (mode == 0 && !dens) xout[(int64_t)d * n + i] = 1.0f / (1.0f + __expf(-y));
            }
            // forward: acc = log |det dx/dz| = -log q; inverse: acc = log q(x)
            if (mode == 1) {
                wout[i] = acc;
            } else if (alpha == 0.f) {
                wout[i] = __expf(acc);
            } else {
                const float q = __expf(dens ? acc : -acc);
                wout[i] = 1.0f / fmaf(1.0f - alpha, q, alpha);
            }
        }
        __syncthreads();   // the next block reuses the coordinate tiles
    }
}

// ---- training: inverse pass with loss and initial gradient -----------------------------
// v = logit(x) through layers K-1..0; L = -sum w_hat log q; dL/dv0 = -(1 - 2 z) w_hat.
// Writes v0 [D][n], g [D][n]; adds its part of the loss to *loss.
__global__ void __launch_bounds__(128) flow_inverse_train_kernel(const unsigned char *__restrict__ wglob, FlowDims f,
                                                                  int64_t n, const float *__restrict__ xin,
                                                                  const float *__restrict__ w,
                                                                  const double *__restrict__ wsum,
                                                                  float *__restrict__ vout, float *__restrict__ gout,
                                                                  float *__restrict__ loss, int *status) {
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char *wsm = smem;
    float *ys = reinterpret_cast<float *>(smem + LAYER_BYTES);
    float *ld = ys + BLOCK * YS;
    uint64_t *bar = reinterpret_cast<uint64_t *>(ld + BLOCK);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, t = lane & 3;
    if (tid == 0) {
        mbar_init(bar, 1);
        fence_mbarrier_init();
    }
    __syncthreads();
    uint32_t phase = 0;
    const float inv_wsum = (float)(1.0 / *wsum);
    const int64_t nblocks = (n + BLOCK - 1) / BLOCK;
    for (int64_t blk = blockIdx.x; blk < nblocks; blk += gridDim.x) {
        const int64_t base = blk * BLOCK;
        for (int r = tid; r < BLOCK; r += blockDim.x) {
            const int64_t i = base + r;
            float acc = 0.f;
            for (int d = 0; d < f.D; ++d) {
                const float x = clamp_unit(i < n ? xin[(int64_t)d * n + i] : 0.5f);
                const float y = __logf(x) - log1pf(-x);
                ys[r * YS + d] = y;
                acc -= log_sig_deriv(y);
            }
            for (int d = f.D; d < YS; ++d) ys[r * YS + d] = 0.f;
            ld[r] = acc;
        }
        for (int step = 0; step < f.K; ++step) {
            const int l = f.K - 1 - step;
            if (!stage_layer(wsm, wglob, l, bar, phase)) {
                if (tid == 0 && status) atomicExch(status, DEV_ST_TIMEOUT);
                return;
            }
            const LayerSmem L = layer_view(wsm);
            for (int r = 0; r < ROUNDS; ++r) {
                float *tile = ys + (size_t)(r * 64 + warp * 16) * YS;
                float *tld = ld + r * 64 + warp * 16;
                uint32_t ain[4], h1a[8][4], h2a[8][4];
                float o[4][4];
                input_frag(tile, f, l, g, t, ain);
                mlp_forward(L, ain, h1a, h2a, o, g, t);
                coupling(tile, tld, f, l, o, g, t, -1.f);
                __syncwarp();
            }
        }
        __syncthreads();
        float part = 0.f;
        for (int r = tid; r < BLOCK; r += blockDim.x) {
            const int64_t i = base + r;
            if (i >= n) continue;
            const float wh = w[i] * inv_wsum;
            float logq = ld[r];
            for (int d = 0; d < f.D; ++d) {
                const float v = ys[r * YS + d];
                logq += log_sig_deriv(v);
                const float z = 1.0f / (1.0f + __expf(-v));
                vout[(int64_t)d * n + i] = v;
                gout[(int64_t)d * n + i] = -(1.0f - 2.0f * z) * wh;
            }
            part -= wh * logq;
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
        if (lane == 0) atomicAdd(loss, part);
        __syncthreads();   // the next block reuses the coordinate tiles
    }
}

// ---- training: backward through one layer ----------------------------------------------
// For layer l (processed in the order 0..K-1 after the inverse pass): recompute
// the MLP on v_A, propagate g through the coupling and the MLP, move v to the
// previous boundary (v_B <- v_B e^s + t) and accumulate the layer's weight
// gradients: dW2 in shared memory (FP32), dW1/dW3/biases in registers and
// shared memory, added to the global FP32 gradient at the end.
constexpr int TPAD = 72;   // padded sample stride of the transposed tiles (64 samples)

struct BwdSmem {
    // byte offsets
    static constexpr int W = 0;
    static constexpr int DW2 = W + LAYER_BYTES;                       // [128][128] f32
    static constexpr int DB = DW2 + H * H * 4;                        // db1[128], db2[128], db3[32] f32
    static constexpr int H1T = DB + (H + H + 32) * 4;                 // [128][TPAD] bf16
    static constexpr int H2T = H1T + H * TPAD * 2;
    static constexpr int GH1T = H2T + H * TPAD * 2;
    static constexpr int GH2T = GH1T + H * TPAD * 2;
    static constexpr int GOT = GH2T + H * TPAD * 2;                   // [32][TPAD]
    static constexpr int AT = GOT + 32 * TPAD * 2;                    // [16][TPAD]
    static constexpr int VT = AT + 16 * TPAD * 2;                     // v, g tiles [64][YS] f32 each
    static constexpr int GT = VT + 64 * YS * 4;
    static constexpr int BAR = GT + 64 * YS * 4;
    static constexpr int TOTAL = BAR + 16;
};

__device__ __forceinline__ void st_bf16(__nv_bfloat16 *base, int row, int col, float v) {
    base[row * TPAD + col] = __float2bfloat16_rn(v);
}

__global__ void __launch_bounds__(128) flow_backward_layer_kernel(const unsigned char *__restrict__ wglob, FlowDims f,
                                                                   int l, int64_t n, const float *__restrict__ w,
                                                                   const double *__restrict__ wsum,
                                                                   float *__restrict__ vbuf, float *__restrict__ gbuf,
                                                                   float *__restrict__ grad_layer, int *status) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, t = lane & 3;
    float *dW2 = reinterpret_cast<float *>(smem + BwdSmem::DW2);
    float *db = reinterpret_cast<float *>(smem + BwdSmem::DB);
    __nv_bfloat16 *h1T = reinterpret_cast<__nv_bfloat16 *>(smem + BwdSmem::H1T);
    __nv_bfloat16 *h2T = reinterpret_cast<__nv_bfloat16 *>(smem + BwdSmem::H2T);
    __nv_bfloat16 *gh1T = reinterpret_cast<__nv_bfloat16 *>(smem + BwdSmem::GH1T);
    __nv_bfloat16 *gh2T = reinterpret_cast<__nv_bfloat16 *>(smem + BwdSmem::GH2T);
    __nv_bfloat16 *goT = reinterpret_cast<__nv_bfloat16 *>(smem + BwdSmem::GOT);
    __nv_bfloat16 *aT = reinterpret_cast<__nv_bfloat16 *>(smem + BwdSmem::AT);
    float *vt = reinterpret_cast<float *>(smem + BwdSmem::VT);
    float *gt = reinterpret_cast<float *>(smem + BwdSmem::GT);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + BwdSmem::BAR);
    for (int k = tid; k < H * H + H + H + 32; k += blockDim.x) {
        if (k < H * H) dW2[k] = 0.f;
        else db[k - H * H] = 0.f;
    }
    if (tid == 0) {
        mbar_init(bar, 1);
        fence_mbarrier_init();
    }
    uint32_t phase = 0;
    if (!stage_layer(smem + BwdSmem::W, wglob, l, bar, phase)) {
        if (tid == 0 && status) atomicExch(status, DEV_ST_TIMEOUT);
        return;
    }
    const LayerSmem L = layer_view(smem + BwdSmem::W);
    const int na = a_size(f, l), nb = b_size(f, l);
    const float inv_wsum = (float)(1.0 / *wsum);
    // register accumulators of dW3 (warp: n-tiles 4w..4w+3, both m-tiles) and dW1 (rows 32w..32w+31)
    float dw3[2][4][4], dw1[2][2][4];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
            for (int q = 0; q < 4; ++q) dw3[a][b][q] = 0.f;
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int q = 0; q < 4; ++q) dw1[a][b][q] = 0.f;

    const int64_t nrounds = (n + 63) / 64;
    for (int64_t rnd = blockIdx.x; rnd < nrounds; rnd += gridDim.x) {
        const int64_t base = rnd * 64;
        // load v and g tiles (64 samples)
        for (int k = tid; k < 64 * YS; k += blockDim.x) {
            const int r = k / YS, d = k % YS;
            const int64_t i = base + r;
            const bool ok = i < n && d < f.D;
            vt[k] = ok ? vbuf[(int64_t)d * n + i] : 0.f;
            gt[k] = ok ? gbuf[(int64_t)d * n + i] : 0.f;
        }
        __syncthreads();
        float *tv = vt + warp * 16 * YS;
        float *tg = gt + warp * 16 * YS;
        const int col0 = warp * 16;       // sample column of this warp in the transposed tiles
        {
            uint32_t ain[4], h1a[8][4], h2a[8][4];
            float o[4][4];
            input_frag(tv, f, l, g, t, ain);
            mlp_forward(L, ain, h1a, h2a, o, g, t);
            // coupling backward (loss weight w_hat per sample row)
            float go[4][4];
#pragma unroll
            for (int half = 0; half < 2; ++half) {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int j = c_col(half, q, t);
                    const int row = c_row(q, g);
                    const int64_t i = base + col0 + row;
                    float gs = 0.f, gtt = 0.f;
                    if (j < nb && i < n) {
                        const float s = S_CLAMP * tanhf(o[half][q] * (1.0f / S_CLAMP));
                        const float tt = o[half + 2][q];
                        const int c = b_idx(f, l, j);
                        const float vB = tv[row * YS + c];
                        const float gB = tg[row * YS + c];
                        const float es = __expf(-s);
                        gtt = -gB * es;
                        const float g_s = -gB * vB + w[i] * inv_wsum;
                        gs = g_s * (1.0f - (s / S_CLAMP) * (s / S_CLAMP));
                        tg[row * YS + c] = gB * es;
                        tv[row * YS + c] = fmaf(vB, __expf(s), tt);
                    }
                    go[half][q] = gs;
                    go[half + 2][q] = gtt;
                }
            }
            // transposed tiles for the weight gradients: a, h1, h2, g_o
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                // a fragment layout: ain regs hold (row, col) pairs of the 16 x 16 input tile
                const int row = (q & 1) ? g + 8 : g;
                const int cc = (q >> 1) * 8 + 2 * t;
                st_bf16(aT, cc, col0 + row, bf_lo(ain[q]));
                st_bf16(aT, cc + 1, col0 + row, bf_hi(ain[q]));
            }
#pragma unroll
            for (int j = 0; j < 8; ++j) {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int row = (q & 1) ? g + 8 : g;
                    const int cc = 16 * j + (q >> 1) * 8 + 2 * t;
                    st_bf16(h1T, cc, col0 + row, bf_lo(h1a[j][q]));
                    st_bf16(h1T, cc + 1, col0 + row, bf_hi(h1a[j][q]));
                    st_bf16(h2T, cc, col0 + row, bf_lo(h2a[j][q]));
                    st_bf16(h2T, cc + 1, col0 + row, bf_hi(h2a[j][q]));
                }
            }
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int row = c_row(q, g);
                    const int cc = nt * 8 + 2 * t + (q & 1);
                    st_bf16(goT, cc, col0 + row, go[nt][q]);
                }
            }
            // g_h2 = g_o W3 (B[k][n] = W3[k][n]), masked by h2 > 0
            uint32_t ga[2][4];
            c_to_a(go[0], go[1], ga[0]);
            c_to_a(go[2], go[3], ga[1]);
            uint32_t gh2a[8][4];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                float c0[4] = {0.f, 0.f, 0.f, 0.f}, c1[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                for (int kt = 0; kt < 2; ++kt) {
                    uint32_t b0, b1;
                    bfrag_t(L.W3, W3_LD, kt, 2 * j, g, t, b0, b1);
                    mma16816(c0, ga[kt], b0, b1);
                    bfrag_t(L.W3, W3_LD, kt, 2 * j + 1, g, t, b0, b1);
                    mma16816(c1, ga[kt], b0, b1);
                }
                // mask: h2a[j] holds h2 at the same positions (reg0 = c0[0..1], reg1 = c0[2..3], ...)
                c0[0] = bf_lo(h2a[j][0]) > 0.f ? c0[0] : 0.f;
                c0[1] = bf_hi(h2a[j][0]) > 0.f ? c0[1] : 0.f;
                c0[2] = bf_lo(h2a[j][1]) > 0.f ? c0[2] : 0.f;
                c0[3] = bf_hi(h2a[j][1]) > 0.f ? c0[3] : 0.f;
                c1[0] = bf_lo(h2a[j][2]) > 0.f ? c1[0] : 0.f;
                c1[1] = bf_hi(h2a[j][2]) > 0.f ? c1[1] : 0.f;
                c1[2] = bf_lo(h2a[j][3]) > 0.f ? c1[2] : 0.f;
                c1[3] = bf_hi(h2a[j][3]) > 0.f ? c1[3] : 0.f;
                c_to_a(c0, c1, gh2a[j]);
            }
            // g_h1 = g_h2 W2 (B[k][n] = W2[k][n]), masked by h1 > 0
            uint32_t gh1a[8][4];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                float c0[4] = {0.f, 0.f, 0.f, 0.f}, c1[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                for (int kt = 0; kt < 8; ++kt) {
                    uint32_t b0, b1;
                    bfrag_t(L.W2, W2_LD, kt, 2 * j, g, t, b0, b1);
                    mma16816(c0, gh2a[kt], b0, b1);
                    bfrag_t(L.W2, W2_LD, kt, 2 * j + 1, g, t, b0, b1);
                    mma16816(c1, gh2a[kt], b0, b1);
                }
                c0[0] = bf_lo(h1a[j][0]) > 0.f ? c0[0] : 0.f;
                c0[1] = bf_hi(h1a[j][0]) > 0.f ? c0[1] : 0.f;
                c0[2] = bf_lo(h1a[j][1]) > 0.f ? c0[2] : 0.f;
                c0[3] = bf_hi(h1a[j][1]) > 0.f ? c0[3] : 0.f;
                c1[0] = bf_lo(h1a[j][2]) > 0.f ? c1[0] : 0.f;
                c1[1] = bf_hi(h1a[j][2]) > 0.f ? c1[1] : 0.f;
                c1[2] = bf_lo(h1a[j][3]) > 0.f ? c1[2] : 0.f;
                c1[3] = bf_hi(h1a[j][3]) > 0.f ? c1[3] : 0.f;
                c_to_a(c0, c1, gh1a[j]);
            }
            // g_a = g_h1 W1 (B[k][n] = W1[k][n]), added to g_A
            float gc[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
#pragma unroll
            for (int kt = 0; kt < 8; ++kt) {
#pragma unroll
                for (int nt = 0; nt < 2; ++nt) {
                    uint32_t b0, b1;
                    bfrag_t(L.W1, W1_LD, kt, nt, g, t, b0, b1);
                    mma16816(gc[nt], gh1a[kt], b0, b1);
                }
            }
#pragma unroll
            for (int nt = 0; nt < 2; ++nt) {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int i = nt * 8 + 2 * t + (q & 1);
                    if (i < na) tg[c_row(q, g) * YS + a_idx(f, l, i)] += gc[nt][q];
                }
            }
            // transposed gradient tiles
#pragma unroll
            for (int j = 0; j < 8; ++j) {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int row = (q & 1) ? g + 8 : g;
                    const int cc = 16 * j + (q >> 1) * 8 + 2 * t;
                    st_bf16(gh1T, cc, col0 + row, bf_lo(gh1a[j][q]));
                    st_bf16(gh1T, cc + 1, col0 + row, bf_hi(gh1a[j][q]));
                    st_bf16(gh2T, cc, col0 + row, bf_lo(gh2a[j][q]));
                    st_bf16(gh2T, cc + 1, col0 + row, bf_hi(gh2a[j][q]));
                }
            }
        }
        __syncthreads();
        // write v, g back
        for (int k = tid; k < 64 * YS; k += blockDim.x) {
            const int r = k / YS, d = k % YS;
            const int64_t i = base + r;
            if (i < n && d < f.D) {
                vbuf[(int64_t)d * n + i] = vt[k];
                gbuf[(int64_t)d * n + i] = gt[k];
            }
        }
        // weight gradients over the 64 samples (K dimension = samples)
        auto afrag_T = [&](const __nv_bfloat16 *T, int m0, int kt, uint32_t (&a)[4]) {
            const __nv_bfloat16 *p = T + (m0 + g) * TPAD + kt * 16 + 2 * t;
            a[0] = *reinterpret_cast<const uint32_t *>(p);
            a[1] = *reinterpret_cast<const uint32_t *>(p + 8 * TPAD);
            a[2] = *reinterpret_cast<const uint32_t *>(p + 8);
            a[3] = *reinterpret_cast<const uint32_t *>(p + 8 * TPAD + 8);
        };
        // dW2[o][i] += sum_s gh2[s][o] h1[s][i]: warp owns rows 32w..32w+31
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
            const int m0 = warp * 32 + mt * 16;
#pragma unroll
            for (int nh = 0; nh < 2; ++nh) {
                float acc[8][4];
#pragma unroll
                for (int a = 0; a < 8; ++a)
#pragma unroll
                    for (int q = 0; q < 4; ++q) acc[a][q] = 0.f;
#pragma unroll
                for (int kt = 0; kt < 4; ++kt) {
                    uint32_t a[4];
                    afrag_T(gh2T, m0, kt, a);
#pragma unroll
                    for (int nn = 0; nn < 8; ++nn) {
                        uint32_t b0, b1;
                        bfrag(h1T, TPAD, kt, nh * 8 + nn, g, t, b0, b1);
                        mma16816(acc[nn], a, b0, b1);
                    }
                }
#pragma unroll
                for (int nn = 0; nn < 8; ++nn) {
                    const int c = (nh * 8 + nn) * 8 + 2 * t;
                    dW2[(m0 + g) * H + c] += acc[nn][0];
                    dW2[(m0 + g) * H + c + 1] += acc[nn][1];
                    dW2[(m0 + g + 8) * H + c] += acc[nn][2];
                    dW2[(m0 + g + 8) * H + c + 1] += acc[nn][3];
                }
            }
        }
        // dW3[o][i] += sum_s go[s][o] h2[s][i]: warp owns n-tiles 4w..4w+3
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
#pragma unroll
            for (int kt = 0; kt < 4; ++kt) {
                uint32_t a[4];
                afrag_T(goT, mt * 16, kt, a);
#pragma unroll
                for (int nn = 0; nn < 4; ++nn) {
                    uint32_t b0, b1;
                    bfrag(h2T, TPAD, kt, warp * 4 + nn, g, t, b0, b1);
                    mma16816(dw3[mt][nn], a, b0, b1);
                }
            }
        }
        // dW1[o][i] += sum_s gh1[s][o] a[s][i]: warp owns rows 32w..32w+31
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
#pragma unroll
            for (int kt = 0; kt < 4; ++kt) {
                uint32_t a[4];
                afrag_T(gh1T, warp * 32 + mt * 16, kt, a);
#pragma unroll
                for (int nn = 0; nn < 2; ++nn) {
                    uint32_t b0, b1;
                    bfrag(aT, TPAD, kt, nn, g, t, b0, b1);
                    mma16816(dw1[mt][nn], a, b0, b1);
                }
            }
        }
        // bias gradients: sums over the 64 sample columns of the transposed tiles
        for (int k = tid; k < H + H + 32; k += blockDim.x) {
            const __nv_bfloat16 *row = k < H ? gh1T + k * TPAD : (k < 2 * H ? gh2T + (k - H) * TPAD : goT + (k - 2 * H) * TPAD);
            float s = 0.f;
            for (int c = 0; c < 64; ++c) s += __bfloat162float(row[c]);
            db[k] += s;
        }
        __syncthreads();
    }
    // flush: global gradient layout of the layer = padded [W1p 128x16 | b1 | W2 128x128 | b2 | W3p 32x128 | b3p]
    float *gW1 = grad_layer;
    float *gb1 = gW1 + H * 16;
    float *gW2 = gb1 + H;
    float *gb2 = gW2 + H * H;
    float *gW3 = gb2 + H;
    float *gb3 = gW3 + 32 * H;
    for (int k = tid; k < H * H; k += blockDim.x) atomicAdd(gW2 + k, dW2[k]);
    for (int k = tid; k < H; k += blockDim.x) {
        atomicAdd(gb1 + k, db[k]);
        atomicAdd(gb2 + k, db[H + k]);
    }
    for (int k = tid; k < 32; k += blockDim.x) atomicAdd(gb3 + k, db[2 * H + k]);
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nn = 0; nn < 4; ++nn) {
            const int r0 = mt * 16 + g, c = (warp * 4 + nn) * 8 + 2 * t;
            atomicAdd(gW3 + r0 * H + c, dw3[mt][nn][0]);
            atomicAdd(gW3 + r0 * H + c + 1, dw3[mt][nn][1]);
            atomicAdd(gW3 + (r0 + 8) * H + c, dw3[mt][nn][2]);
            atomicAdd(gW3 + (r0 + 8) * H + c + 1, dw3[mt][nn][3]);
        }
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nn = 0; nn < 2; ++nn) {
            const int r0 = warp * 32 + mt * 16 + g, c = nn * 8 + 2 * t;
            atomicAdd(gW1 + r0 * 16 + c, dw1[mt][nn][0]);
            atomicAdd(gW1 + r0 * 16 + c + 1, dw1[mt][nn][1]);
            atomicAdd(gW1 + (r0 + 8) * 16 + c, dw1[mt][nn][2]);
            atomicAdd(gW1 + (r0 + 8) * 16 + c + 1, dw1[mt][nn][3]);
        }
}

// ---- parameter plumbing -----------------------------------------------------------------
constexpr int GRAD_LAYER = H * 16 + H + H * H + H + 32 * H + 32;   // padded per-layer gradient floats

struct LayerIdx {
    int a, b;              // half sizes
    int64_t off;           // blob offset of the layer
};

__global__ void pack_weights_kernel(const float *__restrict__ blob, const LayerIdx *__restrict__ li, int K,
                                    unsigned char *__restrict__ wpack) {
    const int l = blockIdx.y;
    if (l >= K) return;
    const LayerIdx L = li[l];
    const float *W1 = blob + L.off;
    const float *b1 = W1 + H * L.a;
    const float *W2 = b1 + H;
    const float *b2 = W2 + H * H;
    const float *W3 = b2 + H;
    const float *b3 = W3 + 2 * L.b * H;
    unsigned char *out = wpack + (size_t)l * LAYER_BYTES;
    __nv_bfloat16 *pW1 = reinterpret_cast<__nv_bfloat16 *>(out + OFF_W1);
    __nv_bfloat16 *pW2 = reinterpret_cast<__nv_bfloat16 *>(out + OFF_W2);
    __nv_bfloat16 *pW3 = reinterpret_cast<__nv_bfloat16 *>(out + OFF_W3);
    float *pb1 = reinterpret_cast<float *>(out + OFF_B1);
    float *pb2 = reinterpret_cast<float *>(out + OFF_B2);
    float *pb3 = reinterpret_cast<float *>(out + OFF_B3);
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < H * W2_LD; k += gridDim.x * blockDim.x) {
        const int r = k / W2_LD, c = k % W2_LD;
        pW2[k] = __float2bfloat16_rn(c < H ? W2[r * H + c] : 0.f);
        if (k < H * W1_LD) {
            const int r1 = k / W1_LD, c1 = k % W1_LD;
            pW1[k] = __float2bfloat16_rn(c1 < L.a ? W1[r1 * L.a + c1] : 0.f);
        }
        if (k < 32 * W3_LD) {
            const int r3 = k / W3_LD, c3 = k % W3_LD;
            float v = 0.f;
            if (c3 < H) {
                if (r3 < 16 && r3 < L.b) v = W3[r3 * H + c3];                       // s rows
                else if (r3 >= 16 && r3 - 16 < L.b) v = W3[(L.b + r3 - 16) * H + c3];  // t rows
            }
            pW3[k] = __float2bfloat16_rn(v);
        }
        if (k < H) {
            pb1[k] = b1[k];
            pb2[k] = b2[k];
        }
        if (k < 32) pb3[k] = (k < 16) ? (k < L.b ? b3[k] : 0.f) : (k - 16 < L.b ? b3[L.b + k - 16] : 0.f);
    }
}

// padded per-layer gradients -> blob layout (overwrites grad_blob)
__global__ void unpack_grad_kernel(const float *__restrict__ gpad, const LayerIdx *__restrict__ li, int K,
                                   float *__restrict__ grad_blob) {
    const int l = blockIdx.y;
    if (l >= K) return;
    const LayerIdx L = li[l];
    const float *gW1 = gpad + (size_t)l * GRAD_LAYER;
    const float *gb1 = gW1 + H * 16;
    const float *gW2 = gb1 + H;
    const float *gb2 = gW2 + H * H;
    const float *gW3 = gb2 + H;
    const float *gb3 = gW3 + 32 * H;
    float *W1 = grad_blob + L.off;
    float *b1 = W1 + H * L.a;
    float *W2 = b1 + H;
    float *b2 = W2 + H * H;
    float *W3 = b2 + H;
    float *b3 = W3 + 2 * L.b * H;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < H * H; k += gridDim.x * blockDim.x) {
        W2[k] = gW2[k];
        if (k < H * L.a) W1[k] = gW1[(k / L.a) * 16 + k % L.a];
        if (k < 2 * L.b * H) {
            const int r = k / H, c = k % H;
            W3[k] = r < L.b ? gW3[r * H + c] : gW3[(16 + r - L.b) * H + c];
        }
        if (k < H) {
            b1[k] = gb1[k];
            b2[k] = gb2[k];
        }
        if (k < 2 * L.b) b3[k] = k < L.b ? gb3[k] : gb3[16 + k - L.b];
    }
}

__global__ void adam_kernel(float *__restrict__ p, const float *__restrict__ gr, float *__restrict__ m,
                            float *__restrict__ v, int64_t n, float lr, float b1t, float b2t) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const float gk = gr[k];
    const float mk = 0.9f * m[k] + 0.1f * gk;
    const float vk = 0.999f * v[k] + 0.001f * gk * gk;
    m[k] = mk;
    v[k] = vk;
    const float mh = mk / (1.0f - b1t);
    const float vh = vk / (1.0f - b2t);
    p[k] -= lr * mh / (sqrtf(vh) + 1e-8f);
}

__global__ void sum_weights_kernel(const float *__restrict__ w, int64_t n, double *__restrict__ out) {
    __shared__ double sh[256];
    double s = 0.0;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        s += (double)w[k];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(out, sh[0]);
}


// ---- tcgen05 (5th-generation tensor core) sampling / density kernel ------------------
// Thread pairs own the rows of 128-sample tiles (row = TMEM lane; the two
// halves of the CTA split every epilogue's columns).  Per layer the three GEMMs
// of the coupling MLP are single-thread-issued tcgen05.mma (kind::f16: BF16 x
// BF16 -> FP32) on operands in shared memory in the no-swizzle K-major
// core-matrix layout (8 rows x 16 bytes per core matrix; LBO = 128 bytes
// between k-chunks, SBO between 8-row groups), with the accumulators in TMEM;
// the epilogues (bias, ReLU, BF16 A operand of the next GEMM) and the affine
// coupling read the rows back with tcgen05.ld.  Two tiles are in flight so that
// one tile's GEMM runs while the threads work on the other's epilogue.  Layer
// weights (46 KB) are staged by 1-D TMA bulk copies into a double buffer, the
// next layer's copy overlapping the current layer.  Same inputs, outputs and
// modes as flow_pass_kernel.
namespace umma {
constexpr int W1B = 128 * 16 * 2;             // W1 [128 n][16 k] BF16
constexpr int W2B = 128 * 128 * 2;            // W2 [128 n][128 k]
constexpr int W3B = 32 * 128 * 2;             // W3 [32 n][128 k]: rows 0..15 s, 16..31 t
constexpr int OFF_W1 = 0, OFF_W2 = OFF_W1 + W1B, OFF_W3 = OFF_W2 + W2B;
constexpr int OFF_B1 = OFF_W3 + W3B, OFF_B2 = OFF_B1 + 128 * 4, OFF_B3 = OFF_B2 + 128 * 4;
constexpr int LAYER = OFF_B3 + 32 * 4;        // 46208 bytes per layer
constexpr int TILES = 4;                      // tiles per block: one weight staging per layer and 512 samples
constexpr int BLOCK_U = 128 * TILES;
constexpr int THREADS = 256;                  // two threads per tile row: column halves of every epilogue
constexpr int YSU = 25;                       // coordinate row stride in floats (odd: no bank conflicts)
constexpr int S_W = 0;                        // shared memory: two layer buffers
constexpr int S_A1 = S_W + 2 * LAYER;         // A of GEMM1 [128][16] (SBO 256), one per tile of a pair
constexpr int S_A2 = S_A1 + 2 * W1B;          // A of GEMM2 / GEMM3 [128][128] (SBO 2048), one per tile of a pair
constexpr int S_Y = S_A2 + 2 * W2B;           // coordinates [BLOCK_U][YSU] f32
constexpr int S_LD = S_Y + BLOCK_U * YSU * 4; // log-Jacobian parts [2][BLOCK_U] (one per column half)
constexpr int S_BAR = S_LD + 2 * BLOCK_U * 4; // weight barriers [2], MMA barriers [2], TMEM address
constexpr int SMEM = S_BAR + 48;
constexpr uint32_t TMEM_COLS = 512;           // per tile of a pair: D1 and D3 at +0, D2 at +128
static_assert(LAYER % 16 == 0 && S_A1 % 16 == 0 && S_A2 % 16 == 0 && S_BAR % 8 == 0, "alignment");
static_assert(SMEM <= 227 * 1024, "shared memory");

// byte offset of element (row, k) in the core-matrix layout with 8-row-group stride sbo
__host__ __device__ __forceinline__ uint32_t core_off(int row, int k, uint32_t sbo) {
    return (uint32_t)(row >> 3) * sbo + (uint32_t)(k >> 3) * 128u + (uint32_t)(row & 7) * 16u + (uint32_t)(k & 7) * 2u;
}
// shared-memory matrix descriptor: start, LBO, SBO (bytes, 16-byte units), version 1, no swizzle
__device__ __forceinline__ uint64_t sdesc(const void *p, uint32_t lbo, uint32_t sbo) {
    const uint32_t a = smem_addr(p);
    return (uint64_t)((a >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
// instruction descriptor, kind::f16: FP32 accumulate, BF16 A and B, both K-major, M = 128
__host__ __device__ constexpr uint32_t idesc(int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}
__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d), "l"(a), "l"(b), "r"(id),
                 "r"(acc)
                 : "memory");
}
__device__ __forceinline__ void commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
                 : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// 32 consecutive FP32 columns of this thread's TMEM lane (asynchronous: wait_ld before use)
__device__ __forceinline__ void ld32_async(uint32_t taddr, uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
          "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
          "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr));
}
__device__ __forceinline__ void wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
// 8 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void ld8(uint32_t taddr, uint32_t (&v)[8]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
                 : "r"(taddr));
    wait_ld();
}
// hidden-layer epilogue for columns [c_lo, c_lo + 64) of this thread's accumulator
// row: + bias, ReLU, BF16 -> that row of A (SBO 2048)
__device__ __forceinline__ void epi_hidden(uint32_t taddr, const float *bias, unsigned char *a, int row, int c_lo) {
    uint32_t v[2][32];
    ld32_async(taddr + (uint32_t)c_lo, v[0]);
    ld32_async(taddr + (uint32_t)c_lo + 32u, v[1]);
    wait_ld();
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int c0 = c_lo + 32 * h;
        uint32_t pk[16];
#pragma unroll
        for (int j = 0; j < 16; ++j)
            pk[j] = relu_pack(__uint_as_float(v[h][2 * j]) + bias[c0 + 2 * j],
                              __uint_as_float(v[h][2 * j + 1]) + bias[c0 + 2 * j + 1]);
#pragma unroll
        for (int q = 0; q < 4; ++q)
            *reinterpret_cast<uint4 *>(a + core_off(row, c0 + 8 * q, 2048)) =
                make_uint4(pk[4 * q], pk[4 * q + 1], pk[4 * q + 2], pk[4 * q + 3]);
    }
}
// S tanh(x / S) from one exponential: S (1 - 2 / (exp(2 x / S) + 1)), saturating to +-S
__device__ __forceinline__ float soft_clamp(float x) {
    const float e = __expf(fminf(fmaxf(x * (2.0f / S_CLAMP), -40.0f), 40.0f));
    return S_CLAMP * (1.0f - __fdividef(2.0f, e + 1.0f));
}
}  // namespace umma

// Weights of every layer in the tcgen05 operand layout (BF16 core matrices) + FP32 biases.
__global__ void pack_umma_kernel(const float *__restrict__ blob, const LayerIdx *__restrict__ li, int K,
                                 unsigned char *__restrict__ wu) {
    const int l = blockIdx.y;
    if (l >= K) return;
    const LayerIdx L = li[l];
    const float *W1 = blob + L.off;
    const float *b1 = W1 + H * L.a;
    const float *W2 = b1 + H;
    const float *b2 = W2 + H * H;
    const float *W3 = b2 + H;
    const float *b3 = W3 + 2 * L.b * H;
    unsigned char *out = wu + (size_t)l * umma::LAYER;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < H * H; k += gridDim.x * blockDim.x) {
        const int r = k / H, c = k % H;
        *reinterpret_cast<__nv_bfloat16 *>(out + umma::OFF_W2 + umma::core_off(r, c, 2048)) =
            __float2bfloat16_rn(W2[r * H + c]);
        if (k < H * 16) {
            // columns [0, a): W1; 12, 13: b2 as BF16 hi + lo; 14, 15: b1 as hi + lo
            // (a <= 12; the warp-specialised kernel adds the biases on the tensor
            // core through these columns, the other kernels read the FP32 biases)
            const int r1 = k / 16, c1 = k % 16;
            float v = c1 < L.a ? W1[r1 * L.a + c1] : 0.f;
            if (c1 >= 12) {
                const float b = c1 < 14 ? b2[r1] : b1[r1];
                const float hi = __bfloat162float(__float2bfloat16_rn(b));
                v = (c1 & 1) ? b - hi : hi;
            }
            *reinterpret_cast<__nv_bfloat16 *>(out + umma::OFF_W1 + umma::core_off(r1, c1, 256)) =
                __float2bfloat16_rn(v);
        }
        if (k < 32 * H) {
            const int r3 = k / H, c3 = k % H;
            float v = 0.f;
            if (r3 < 16 && r3 < L.b) v = W3[r3 * H + c3];                       // s rows
            else if (r3 >= 16 && r3 - 16 < L.b) v = W3[(L.b + r3 - 16) * H + c3];  // t rows
            *reinterpret_cast<__nv_bfloat16 *>(out + umma::OFF_W3 + umma::core_off(r3, c3, 2048)) =
                __float2bfloat16_rn(v);
        }
        if (k < H) {
            reinterpret_cast<float *>(out + umma::OFF_B1)[k] = b1[k];
            reinterpret_cast<float *>(out + umma::OFF_B2)[k] = b2[k];
        }
        if (k < 32)
            reinterpret_cast<float *>(out + umma::OFF_B3)[k] =
                (k < 16) ? (k < L.b ? b3[k] : 0.f) : (k - 16 < L.b ? b3[L.b + k - 16] : 0.f);
    }
}

__global__ void __launch_bounds__(umma::THREADS, 1) flow_umma_kernel(
    const unsigned char *__restrict__ wglob, FlowDims f, int mode, int64_t n, uint32_t seed_lo, uint32_t seed_hi,
    uint32_t iter, uint32_t inst, const float *__restrict__ xin, float *__restrict__ xout, float *__restrict__ wout,
    int *status, int64_t n_flow, float alpha) {
    using umma::BLOCK_U;
    using umma::LAYER;
    using umma::TILES;
    using umma::YSU;
    using umma::core_off;
    using umma::sdesc;
    using umma::idesc;
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char *wb[2] = {smem + umma::S_W, smem + umma::S_W + LAYER};
    unsigned char *a1[2] = {smem + umma::S_A1, smem + umma::S_A1 + umma::W1B};
    unsigned char *a2[2] = {smem + umma::S_A2, smem + umma::S_A2 + umma::W2B};
    float *ys = reinterpret_cast<float *>(smem + umma::S_Y);
    float *ldj[2] = {reinterpret_cast<float *>(smem + umma::S_LD),
                     reinterpret_cast<float *>(smem + umma::S_LD) + BLOCK_U};
    uint64_t *wbar = reinterpret_cast<uint64_t *>(smem + umma::S_BAR);
    uint64_t *mbar = wbar + 2;
    uint32_t *slot = reinterpret_cast<uint32_t *>(wbar + 4);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int half = warp >> 2;                    // column half of every epilogue
    const int row = (warp & 3) * 32 + (tid & 31);  // tile row = TMEM lane
    if (tid == 0) {
        for (int k = 0; k < 4; ++k) mbar_init(&wbar[k], 1);
        fence_mbarrier_init();
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(slot)),
                     "r"(umma::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    umma::fence_before();
    __syncthreads();
    umma::fence_after();
    const uint32_t tmem = *slot;
    const uint32_t lane = tmem + ((uint32_t)((warp & 3) * 32) << 16);
    const int64_t nblocks = (n + BLOCK_U - 1) / BLOCK_U;
    auto dens_of = [&](int64_t b) { return mode == 1 || b * BLOCK_U >= n_flow; };
    auto layer_of = [&](bool d, int step) { return d ? f.K - 1 - step : step; };
    auto stage = [&](int buf, int l) {   // thread 0: TMA of layer l into buffer buf
        fence_proxy_async_smem();
        mbar_expect_tx(&wbar[buf], LAYER);
        bulk_g2s(wb[buf], wglob + (size_t)l * LAYER, LAYER, &wbar[buf]);
    };
    uint32_t wph[2] = {0u, 0u}, mph[2] = {0u, 0u};
    bool wpending[2] = {false, false}, mpending[2] = {false, false}, failed = false, lfail = false;
    int64_t blk = blockIdx.x;
    if (tid == 0 && blk < nblocks) stage(0, layer_of(dens_of(blk), 0));
    wpending[0] = blk < nblocks;
    // generic shared-memory writes made visible to the tensor core, then a block
    // barrier that also agrees on failure; true when every thread is healthy
    auto publish = [&]() {
        fence_proxy_async_smem();
        umma::fence_before();
        const bool bad = __syncthreads_or(lfail);
        umma::fence_after();
        if (bad) failed = true;
        return !bad;
    };
    // wait for the MMAs committed to barrier p (a thread that gives up reports at the next barrier)
    auto wait_mma = [&](int p) {
        if (mbar_wait_bounded(&mbar[p], mph[p] & 1u, WAIT_LIMIT)) {
            ++mph[p];
            mpending[p] = false;
        } else {
            lfail = true;
        }
        umma::fence_after();
    };
    auto issue = [&](int p) {
        umma::commit(&mbar[p]);
        mpending[p] = true;
    };
    int gstep = 0;
    for (; blk < nblocks && !failed; blk += gridDim.x) {
        const int64_t base = blk * BLOCK_U;
        const bool dens = dens_of(blk);
        // coordinates of the block's samples: rows t * 128 + row, tiles split between the halves
        for (int t = half; t < TILES; t += 2) {
            const int r = t * 128 + row;
            const int64_t i = base + r;
            const bool valid = i < n;
            float acc = 0.f;
            float *y = ys + r * YSU;
            const int64_t ii = valid ? i : base;
            if (mode == 0) {
                const uint32_t c0 = (uint32_t)(uint64_t)ii, c1 = (uint32_t)((uint64_t)ii >> 32);
                for (int blk4 = 0; 4 * blk4 < f.D; ++blk4) {
                    const u32x4 rr = philox4x32_10(u32x4{c0, c1, iter, (inst << 8) | (uint32_t)blk4}, seed_lo, seed_hi);
                    const uint32_t wv[4] = {rr.x, rr.y, rr.z, rr.w};
                    for (int q = 0; q < 4 && 4 * blk4 + q < f.D; ++q) {
                        const float z = word_to_uniform(wv[q]);
                        const float yy = __logf(z) - log1pf(-z);
                        y[4 * blk4 + q] = yy;
                        acc -= log_sig_deriv(yy);
                        // defensive share: the uniform point itself is the sample
                        if (dens && valid) xout[(int64_t)(4 * blk4 + q) * n + i] = z;
                    }
                }
            } else {
                for (int d = 0; d < f.D; ++d) {
                    const float x = clamp_unit(valid ? xin[(int64_t)d * n + i] : 0.5f);
                    const float yy = __logf(x) - log1pf(-x);
                    y[d] = yy;
                    acc -= log_sig_deriv(yy);
                }
            }
            ldj[0][r] = acc;
            ldj[1][r] = 0.f;
        }
        for (int step = 0; step < f.K && !failed; ++step, ++gstep) {
            const int b = gstep & 1;
            const int l = layer_of(dens, step);
            // everyone is done with the other buffer (previous layer): prefetch into it
            __syncthreads();
            int nl = -1;
            if (step + 1 < f.K) nl = layer_of(dens, step + 1);
            else if (blk + gridDim.x < nblocks) nl = layer_of(dens_of(blk + gridDim.x), 0);
            if (nl >= 0) {
                if (tid == 0) stage(b ^ 1, nl);
                wpending[b ^ 1] = true;
            }
            const bool ok = mbar_wait_bounded(&wbar[b], wph[b] & 1u, WAIT_LIMIT);
            if (__syncthreads_or(!ok)) {
                failed = true;
                break;
            }
            ++wph[b];
            wpending[b] = false;
            const unsigned char *W = wb[b];
            const float *b1 = reinterpret_cast<const float *>(W + umma::OFF_B1);
            const float *b2 = reinterpret_cast<const float *>(W + umma::OFF_B2);
            const float *b3 = reinterpret_cast<const float *>(W + umma::OFF_B3);
            const int na = a_size(f, l), nb = b_size(f, l);
            const float dir = dens ? -1.f : 1.f;
            const uint64_t dW1 = sdesc(W + umma::OFF_W1, 128, 256);
            // tiles in pairs: while the threads run one tile's epilogue, the
            // tensor core runs the other tile's GEMM
            for (int t0 = 0; t0 < TILES && !failed; t0 += 2) {
                // A of GEMM1 for both tiles: k chunk `half` of this row's conditioning half
#pragma unroll
                for (int p = 0; p < 2; ++p) {
                    const float *y = ys + ((t0 + p) * 128 + row) * YSU;
                    uint32_t pk[4];
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int k0 = 8 * half + 2 * i;
                        const float v0 = k0 < na ? y[a_idx(f, l, k0)] : 0.f;
                        const float v1 = k0 + 1 < na ? y[a_idx(f, l, k0 + 1)] : 0.f;
                        pk[i] = pack_bf16(v0, v1);
                    }
                    *reinterpret_cast<uint4 *>(a1[p] + core_off(row, 8 * half, 256)) =
                        make_uint4(pk[0], pk[1], pk[2], pk[3]);
                }
                if (!publish()) break;
                if (tid == 0) {
                    for (int p = 0; p < 2; ++p) {
                        umma::mma(tmem + 256 * p, sdesc(a1[p], 128, 256), dW1, idesc(128), 0u);
                        issue(p);
                    }
                }
                // GEMM2 of each tile once its hidden layer 1 is written
                for (int p = 0; p < 2; ++p) {
                    wait_mma(p);
                    umma::epi_hidden(lane + 256 * p, b1, a2[p], row, 64 * half);
                    if (!publish()) break;
                    if (tid == 0) {
#pragma unroll
                        for (int s2 = 0; s2 < 8; ++s2)
                            umma::mma(tmem + 256 * p + 128, sdesc(a2[p] + s2 * 256, 128, 2048),
                                      sdesc(W + umma::OFF_W2 + s2 * 256, 128, 2048), idesc(128), s2 > 0 ? 1u : 0u);
                        issue(p);
                    }
                }
                if (failed) break;
                // GEMM3 (into the tile's first 32 columns: hidden layer 1 is consumed)
                for (int p = 0; p < 2; ++p) {
                    wait_mma(p);
                    umma::epi_hidden(lane + 256 * p + 128, b2, a2[p], row, 64 * half);
                    if (!publish()) break;
                    if (tid == 0) {
#pragma unroll
                        for (int s2 = 0; s2 < 8; ++s2)
                            umma::mma(tmem + 256 * p, sdesc(a2[p] + s2 * 256, 128, 2048),
                                      sdesc(W + umma::OFF_W3 + s2 * 256, 128, 2048), idesc(32), s2 > 0 ? 1u : 0u);
                        issue(p);
                    }
                }
                if (failed) break;
                // affine coupling: this thread's half of the pairs (s, t), j in [8 half, 8 half + 8)
                for (int p = 0; p < 2; ++p) {
                    wait_mma(p);
                    // tcgen05.ld is warp-collective: a warp with a failed wait skips as a whole
                    if (__any_sync(0xffffffffu, lfail)) {
                        lfail = true;
                        continue;
                    }
                    const int r = (t0 + p) * 128 + row;
                    float *y = ys + r * YSU;
                    uint32_t os[8], ot[8];
                    umma::ld8(lane + 256 * p + 8 * half, os);
                    umma::ld8(lane + 256 * p + 16 + 8 * half, ot);
                    float part = 0.f;
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const int j = 8 * half + q;
                        if (j < nb) {
                            const float sv = umma::soft_clamp(__uint_as_float(os[q]) + b3[j]);
                            const float tt = __uint_as_float(ot[q]) + b3[16 + j];
                            float &yy = y[b_idx(f, l, j)];
                            yy = dir > 0.f ? fmaf(yy, __expf(sv), tt) : (yy - tt) * __expf(-sv);
                            part += sv;
                        }
                    }
                    ldj[half][r] += dir * part;
                }
            }
            // rows of the next layer's A come from both halves' couplings
            if (__syncthreads_or(lfail)) failed = true;
        }
        if (failed) break;
        __syncthreads();
        // outputs of the block (tiles split between the halves)
        for (int t = half; t < TILES; t += 2) {
            const int r = t * 128 + row;
            const int64_t i = base + r;
            if (i >= n) continue;
            const float *y = ys + r * YSU;
            float acc = ldj[0][r] + ldj[1][r];
            for (int d = 0; d < f.D; ++d) {
                acc += log_sig_deriv(y[d]);
                if (mode == 0 && !dens) xout[(int64_t)d * n + i] = 1.0f / (1.0f + __expf(-y[d]));
            }
            if (mode == 1) {
                wout[i] = acc;
            } else if (alpha == 0.f) {
                wout[i] = __expf(acc);
            } else {
                const float q = __expf(dens ? acc : -acc);
                wout[i] = 1.0f / fmaf(1.0f - alpha, q, alpha);
            }
        }
    }
    if (failed) {
        // report, let copies and MMAs in flight finish (bounded), then release TMEM
        if (tid == 0 && status) atomicExch(status, DEV_ST_TIMEOUT);
        for (int k = 0; k < 2; ++k) {
            if (wpending[k]) (void)mbar_wait_bounded(&wbar[k], wph[k] & 1u, WAIT_LIMIT);
            if (mpending[k]) (void)mbar_wait_bounded(&mbar[k], mph[k] & 1u, WAIT_LIMIT);
        }
    }
    umma::fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(umma::TMEM_COLS)
                     : "memory");
}


// ---- warp-specialised tcgen05 sampling / density kernel (the default path) -------------
// Roles within a CTA (one CTA per SM):
//   * epilogue warps 0 .. 4 S - 1: slot s = warp / 4 owns one 128-sample tile
//     of the current group; warp % 4 selects the warp's 32 TMEM lanes (tile
//     rows), so every thread owns one sample, whose coordinates stay in
//     registers through all layers;
//   * warp 4 S: one thread issues the slots' GEMMs (tcgen05.mma, kind::f16:
//     BF16 operands in shared memory in the no-swizzle K-major core-matrix
//     layout, FP32 accumulators in TMEM) and owns the TMEM allocation;
//   * warp 4 S + 1: one thread streams the layers' weights (bulk copies into a
//     double buffer, the next layer's copy overlapping the current layer).
// Per layer and slot: GEMM1 (A = the conditioning half, K = 16; b1 enters
// through two columns of ones) -> ReLU, BF16 -> GEMM2 (a K = 16 step that
// puts b2 into the accumulator, then K = 128) -> ReLU, BF16 -> GEMM3
// (N = 32: s | t) -> affine coupling.  Each hand-off goes through one mbarrier
// per direction and slot (a_full: the slot's A operand is written and its
// accumulator read; d_full: the slot's GEMM has completed); the slot's 128
// accumulator columns serve all three GEMMs.  The MMA thread issues the
// slots' GEMMs stage by stage in slot order, so while one slot's warps run an
// epilogue the tensor core runs the other slots' GEMMs.  Same inputs,
// outputs and modes as flow_pass_kernel; every wait is bounded, a timeout is
// reported through the status word, and then every role leaves its loop and
// TMEM is freed.
namespace ws {
constexpr uint32_t tmem_cols(int c) { return c <= 32 ? 32u : c <= 64 ? 64u : c <= 128 ? 128u : c <= 256 ? 256u : 512u; }

// A slot's operand buffer holds, at different times, the A of GEMM2 / GEMM3
// ([128][128], from the hidden epilogues) and the A of GEMM1 ([128][16], at
// offset 0, written by the coupling after GEMM3 has completed and read before
// the next hidden epilogue writes) together with the row scratch (from
// SCRATCH: a thread's coordinates by dimension between groups).
constexpr int A_BYTES = umma::W2B;
constexpr int SCRATCH = umma::W1B;
constexpr int ROW_FLOATS = 33;   // odd: conflict-free rows
static_assert(SCRATCH + 128 * ROW_FLOATS * 4 <= A_BYTES, "GEMM1 operand and row scratch fit a slot's buffer");

template <int S_, int CW_>
struct Cfg {
    static constexpr int S = S_;                          // tiles in flight (slots)
    static constexpr int CW = CW_;                        // hidden columns per TMEM wait
    static constexpr int GROUP = 128 * S;                 // samples per group: all slots run the same layers
    static constexpr int EPI_WARPS = 4 * S;
    static constexpr int MMA_WARP = EPI_WARPS, LOAD_WARP = EPI_WARPS + 1;
    static constexpr int THREADS = 32 * (EPI_WARPS + 2);
    static constexpr int NE = 12;                         // coordinate pairs per half (dim <= 24)
    static constexpr int S_W = 0;                         // two layer buffers
    static constexpr int S_ONES = S_W + 2 * umma::LAYER;  // A of GEMM2's bias step [128][16]
    static constexpr int S_A = S_ONES + umma::W1B;        // per slot: the A operands (A_BYTES)
    static constexpr int S_BAR = S_A + S * A_BYTES;       // a_full[S], d_full[S], wfull[2], wempty[2], mdone
    static constexpr int N_BAR = 2 * S + 5;
    static constexpr int S_MISC = S_BAR + 8 * N_BAR;      // TMEM address, failure flag
    static constexpr int SMEM = S_MISC + 16;
    static constexpr uint32_t TMEM_COLS = tmem_cols(128 * S);
    static constexpr uint32_t A_COUNT = 128;              // a_full: every thread of the slot arrives
    static constexpr uint32_t E_COUNT = 1 + 128 * S;      // wempty: the MMA commit + every epilogue thread
    static_assert(S_ONES % 128 == 0 && S_A % 128 == 0 && S_BAR % 8 == 0, "alignment");
    static_assert(SMEM <= 227 * 1024, "shared memory");
    static_assert(128 * S <= 512, "TMEM columns");
    static_assert(CW == 16 || CW % 32 == 0, "whole TMEM loads per wait");
};
using Default = Cfg<4, 16>;

__device__ __forceinline__ void arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// every lane waits for completion k of `bar` (bounded); the warp agrees on the outcome
__device__ __forceinline__ bool wait_warp(uint64_t *bar, uint32_t k) {
    const bool ok = mbar_wait_bounded(bar, k & 1u, WAIT_LIMIT);
    return __all_sync(0xffffffffu, ok);
}

// 16 consecutive FP32 columns of this thread's TMEM lane (asynchronous: wait_ld before use)
__device__ __forceinline__ void ld16_async(uint32_t taddr, uint32_t *v) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
          "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr));
}

// y = logit(z) and log(z (1 - z)) = log |dz/dy|, from two logarithms
// (1 - z is exact for z >= 1/2)
__device__ __forceinline__ float logit_lsd(float z, float &lsd) {
    const float a = __logf(z), b = __logf(1.0f - z);
    lsd = a + b;
    return a - b;
}
// x = sigmoid(y) and log(x (1 - x)) = -|y| - 2 log(1 + exp(-|y|))
__device__ __forceinline__ float sigmoid_lsd(float y, float &lsd) {
    const float ay = fabsf(y), e = __expf(-ay), r = __fdividef(1.0f, 1.0f + e);
    lsd = -ay - 2.0f * __logf(1.0f + e);
    return y >= 0.f ? r : e * r;
}

// hidden-layer epilogue of this thread's accumulator row (the bias is already
// in it): ReLU, BF16 -> that row of the slot's A operand (SBO 2048), CW
// columns per TMEM wait
template <int CW>
__device__ __forceinline__ void hidden(uint32_t taddr, unsigned char *a, int row) {
    constexpr int LW = CW < 32 ? CW : 32;   // columns per TMEM load
#pragma unroll
    for (int h = 0; h < 128 / CW; ++h) {
        const int c0 = CW * h;
        uint32_t v[CW];
#pragma unroll
        for (int g = 0; g < CW / LW; ++g) {
            if constexpr (LW == 32) umma::ld32_async(taddr + (uint32_t)(c0 + 32 * g), *reinterpret_cast<uint32_t(*)[32]>(v + 32 * g));
            else ld16_async(taddr + (uint32_t)(c0 + 16 * g), v + 16 * g);
        }
        umma::wait_ld();
#pragma unroll
        for (int q = 0; q < CW / 8; ++q) {
            const uint32_t *u = v + 8 * q;
            *reinterpret_cast<uint4 *>(a + umma::core_off(row, c0 + 8 * q, 2048)) =
                make_uint4(relu_pack(__uint_as_float(u[0]), __uint_as_float(u[1])),
                           relu_pack(__uint_as_float(u[2]), __uint_as_float(u[3])),
                           relu_pack(__uint_as_float(u[4]), __uint_as_float(u[5])),
                           relu_pack(__uint_as_float(u[6]), __uint_as_float(u[7])));
        }
    }
}

// One layer for this thread's row.  c: the conditioning half, t: the half the
// coupling transforms (forward: t e^s + shift; inverse: (t - shift) e^-s).
// kd counts the completions of the slot's d_full consumed so far.  Returns
// false (warp-uniform) when a wait gave up.
template <int CW, int NE>
__device__ __forceinline__ bool epi_layer(float (&c)[NE], float (&t)[NE], int na, int nb, bool fwd, float &acc,
                                          const unsigned char *W, unsigned char *a, int row, uint32_t taddr,
                                          uint64_t *a_full, uint64_t *d_full, uint64_t *wempty, uint32_t &kd) {
    const float *b3 = reinterpret_cast<const float *>(W + umma::OFF_B3);
    // GEMM1 operand row: the conditioning half below na, 1 in columns 14 and 15
    // (W1's b1 hi and lo), else 0 (the accumulator's previous contents were read
    // before: wait_ld)
    auto a1v = [&](int k) { return k < NE && k < na ? c[k < NE ? k : 0] : k >= 14 ? 1.0f : 0.f; };
    uint32_t pk[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) pk[k] = pack_bf16(a1v(2 * k), a1v(2 * k + 1));
    *reinterpret_cast<uint4 *>(a + umma::core_off(row, 0, 256)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
    *reinterpret_cast<uint4 *>(a + umma::core_off(row, 8, 256)) = make_uint4(pk[4], pk[5], pk[6], pk[7]);
    fence_proxy_async_smem();
    umma::fence_before();
    arrive(a_full);
    if (!wait_warp(d_full, kd++)) return false;
    umma::fence_after();
    hidden<CW>(taddr, a, row);
    fence_proxy_async_smem();
    umma::fence_before();
    arrive(a_full);
    if (!wait_warp(d_full, kd++)) return false;
    umma::fence_after();
    hidden<CW>(taddr, a, row);
    fence_proxy_async_smem();
    umma::fence_before();
    arrive(a_full);
    if (!wait_warp(d_full, kd++)) return false;
    umma::fence_after();
    // GEMM3: s in columns j, the shift in columns 16 + j (j < nb <= 12)
    uint32_t os[16], ot[16];
    ld16_async(taddr, os);
    ld16_async(taddr + 16u, ot);
    umma::wait_ld();
    float part = 0.f;
#pragma unroll
    for (int j = 0; j < NE; ++j) {
        if (j >= nb) break;   // uniform over the CTA
        const float sv = umma::soft_clamp(__uint_as_float(os[j]) + b3[j]);
        const float sh = __uint_as_float(ot[j]) + b3[16 + j];
        t[j] = fwd ? fmaf(t[j], __expf(sv), sh) : (t[j] - sh) * __expf(-sv);
        part += sv;
    }
    acc += fwd ? part : -part;
    arrive(wempty);   // this thread is done with the layer's weight buffer
    return true;
}

// the GEMM of `stage` (0, 1, 2) for one slot, issued by the MMA thread.
// GEMM1 takes b1 through columns 14, 15 of its operands; GEMM2 starts with
// D = ones x W1^T, the ones tile selecting W1's columns 12, 13 (b2 hi and lo).
__device__ __forceinline__ void issue_stage(int stage, uint32_t d, const unsigned char *W, const unsigned char *a,
                                            const unsigned char *ones) {
    if (stage == 0) {
        umma::mma(d, umma::sdesc(a, 128, 256), umma::sdesc(W + umma::OFF_W1, 128, 256), umma::idesc(128), 0u);
    } else {
        const unsigned char *wb = W + (stage == 1 ? umma::OFF_W2 : umma::OFF_W3);
        const uint32_t id = stage == 1 ? umma::idesc(128) : umma::idesc(32);
        if (stage == 1)
            umma::mma(d, umma::sdesc(ones, 128, 256), umma::sdesc(W + umma::OFF_W1, 128, 256), id, 0u);
#pragma unroll
        for (int ks = 0; ks < 8; ++ks)
            umma::mma(d, umma::sdesc(a + ks * 256, 128, 2048), umma::sdesc(wb + ks * 256, 128, 2048), id,
                      (ks > 0 || stage == 1) ? 1u : 0u);
    }
}
}  // namespace ws

template <class C>
__global__ void __launch_bounds__(C::THREADS, 1) flow_ws_kernel(
    const unsigned char *__restrict__ wglob, FlowDims f, int mode, int64_t n, uint32_t seed_lo, uint32_t seed_hi,
    uint32_t iter, uint32_t inst, const float *__restrict__ xin, float *__restrict__ xout, float *__restrict__ wout,
    int *status, int64_t n_flow, float alpha) {
    constexpr int S = C::S, NE = C::NE;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + C::S_BAR);
    uint64_t *a_full = bars, *d_full = bars + S, *wfull = bars + 2 * S, *wempty = bars + 2 * S + 2;
    uint64_t *mdone = bars + 2 * S + 4;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(smem + C::S_MISC);
    volatile int *fail = reinterpret_cast<volatile int *>(smem + C::S_MISC + 4);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&a_full[s], C::A_COUNT);
            mbar_init(&d_full[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&wfull[b], 1);
            mbar_init(&wempty[b], C::E_COUNT);
        }
        mbar_init(mdone, 1);
        *fail = 0;
        fence_mbarrier_init();
    }
    // the ones tile of GEMM2's bias step: 1 in columns 12 and 13 of every row
    for (int r = tid; r < 128; r += C::THREADS) {
        const uint32_t one2 = pack_bf16(1.0f, 1.0f);
        *reinterpret_cast<uint4 *>(smem + C::S_ONES + umma::core_off(r, 0, 256)) = make_uint4(0u, 0u, 0u, 0u);
        *reinterpret_cast<uint4 *>(smem + C::S_ONES + umma::core_off(r, 8, 256)) = make_uint4(0u, 0u, one2, 0u);
    }
    fence_proxy_async_smem();
    if (warp == C::MMA_WARP) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tslot)),
                     "r"(C::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    umma::fence_before();
    __syncthreads();
    umma::fence_after();
    const uint32_t tmem = *tslot;
    const int64_t ngroups = (n + C::GROUP - 1) / C::GROUP;
    const int64_t my_groups = ngroups > (int64_t)blockIdx.x ? (ngroups - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    auto dens_of = [&](int64_t g) { return mode == 1 || g * C::GROUP >= n_flow; };
    auto give_up = [&]() {
        *fail = 1;
        if (status) atomicExch(status, DEV_ST_TIMEOUT);
    };

    if (warp < C::EPI_WARPS) {
        // ---- epilogue: slot s, TMEM lanes 32 (warp % 4) ..., one sample per lane
        const int s = warp >> 2, row = 32 * (warp & 3) + lane;
        const uint32_t taddr = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + 128u * (uint32_t)s;
        unsigned char *a = smem + C::S_A + s * ws::A_BYTES;
        float *scratch = reinterpret_cast<float *>(a + ws::SCRATCH) + row * ws::ROW_FLOATS;
        const int h = f.h, D = f.D;
        uint32_t kd = 0;
        int64_t gs = 0;
        bool ok = true;
        for (int64_t k = 0; k < my_groups && ok; ++k) {
            if (__any_sync(0xffffffffu, *fail != 0)) {
                ok = false;
                break;
            }
            const int64_t g = blockIdx.x + k * gridDim.x;
            const int64_t base = g * C::GROUP;
            const int64_t i = base + s * 128 + row;
            const bool valid = i < n;
            const bool dens = dens_of(g);
            const int64_t ii = valid ? i : base;
            float acc = 0.f;
            // the row's coordinates y = logit(x), by dimension into the scratch row
            if (mode == 0) {
                const uint32_t c0 = (uint32_t)(uint64_t)ii, c1 = (uint32_t)((uint64_t)ii >> 32);
                for (int b4 = 0; 4 * b4 < D; ++b4) {
                    const u32x4 rr = philox4x32_10(u32x4{c0, c1, iter, (inst << 8) | (uint32_t)b4}, seed_lo, seed_hi);
                    const uint32_t wv[4] = {rr.x, rr.y, rr.z, rr.w};
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int d = 4 * b4 + q;
                        if (d < D) {
                            const float z = word_to_uniform(wv[q]);
                            float lsd;
                            scratch[d] = ws::logit_lsd(z, lsd);
                            acc -= lsd;
                            // defensive share: the uniform point itself is the sample
                            if (dens && valid) xout[(int64_t)d * n + i] = z;
                        }
                    }
                }
            } else {
                // all loads of the row issued before the first use
                float xv[2 * NE];
#pragma unroll
                for (int q = 0; q < 2 * NE; ++q) xv[q] = valid && q < D ? xin[(int64_t)q * n + i] : 0.5f;
#pragma unroll
                for (int q = 0; q < 2 * NE; ++q) {
                    if (q < D) {
                        float lsd;
                        scratch[q] = ws::logit_lsd(clamp_unit(xv[q]), lsd);
                        acc -= lsd;
                    }
                }
            }
            // cnd / trn: the conditioning and the transformed half of the current
            // layer (the first h coordinates for an even layer, the rest for an
            // odd one), swapped after every layer: one copy of the layer code
            const int l0 = dens ? f.K - 1 : 0;
            const int hc = (l0 & 1) ? h : 0, ht = (l0 & 1) ? 0 : h;   // offsets of cnd and trn in the row
            float cnd[NE], trn[NE];
#pragma unroll
            for (int q = 0; q < NE; ++q) {
                cnd[q] = q < ((l0 & 1) ? D - h : h) ? scratch[hc + q] : 0.f;
                trn[q] = q < ((l0 & 1) ? h : D - h) ? scratch[ht + q] : 0.f;
            }
            for (int step = 0; step < f.K; ++step, ++gs) {
                const int l = dens ? f.K - 1 - step : step;
                const int b = (int)(gs & 1);
                if (!ws::wait_warp(&wfull[b], (uint32_t)(gs >> 1))) {
                    ok = false;
                    break;
                }
                if (!ws::epi_layer<C::CW, NE>(cnd, trn, a_size(f, l), b_size(f, l), !dens, acc,
                                              smem + C::S_W + b * umma::LAYER, a, row, taddr, &a_full[s], &d_full[s],
                                              &wempty[b], kd)) {
                    ok = false;
                    break;
                }
#pragma unroll
                for (int q = 0; q < NE; ++q) {
                    const float tq = cnd[q];
                    cnd[q] = trn[q];
                    trn[q] = tq;
                }
            }
            if (!ok) break;
            // after K layers cnd is the half a layer of parity l0 + K would
            // condition on; back into the scratch row by dimension (the slot's
            // last GEMM has completed)
            const bool odd = (l0 + f.K) & 1;
#pragma unroll
            for (int q = 0; q < NE; ++q) {
                if (q < (odd ? D - h : h)) scratch[(odd ? h : 0) + q] = cnd[q];
                if (q < (odd ? h : D - h)) scratch[(odd ? 0 : h) + q] = trn[q];
            }
            if (valid) {
                for (int d = 0; d < D; ++d) {
                    float lsd;
                    const float x = ws::sigmoid_lsd(scratch[d], lsd);
                    acc += lsd;
                    if (mode == 0 && !dens) xout[(int64_t)d * n + i] = x;
                }
                // forward: acc = log |det dx/dz| = -log q; inverse: acc = log q(x)
                if (mode == 1) {
                    wout[i] = acc;
                } else if (alpha == 0.f) {
                    wout[i] = __expf(acc);
                } else {
                    const float q = __expf(dens ? acc : -acc);
                    wout[i] = 1.0f / fmaf(1.0f - alpha, q, alpha);
                }
            }
        }
        if (!ok) give_up();
    } else if (warp == C::MMA_WARP) {
        // ---- MMA issue, in the slots' common order: stage by stage, slot by slot
        if (lane == 0) {
            uint32_t ka[S];
#pragma unroll
            for (int s = 0; s < S; ++s) ka[s] = 0;
            int64_t gs = 0;
            bool ok = true;
            for (int64_t k = 0; k < my_groups && ok; ++k) {
                for (int step = 0; step < f.K; ++step, ++gs) {
                    const int b = (int)(gs & 1);
                    if (!mbar_wait_bounded(&wfull[b], (uint32_t)(gs >> 1) & 1u, WAIT_LIMIT)) {
                        ok = false;
                        break;
                    }
                    const unsigned char *W = smem + C::S_W + b * umma::LAYER;
                    for (int st = 0; st < 3 && ok; ++st) {
#pragma unroll
                        for (int s = 0; s < S; ++s) {
                            if (!mbar_wait_bounded(&a_full[s], ka[s] & 1u, WAIT_LIMIT)) {
                                ok = false;
                                break;
                            }
                            ++ka[s];
                            umma::fence_after();
                            ws::issue_stage(st, tmem + 128u * (uint32_t)s, W, smem + C::S_A + s * ws::A_BYTES,
                                            smem + C::S_ONES);
                            umma::commit(&d_full[s]);
                        }
                    }
                    if (!ok) break;
                    // the weight buffer is free once every slot's last GEMM of the step has completed
                    umma::commit(&wempty[b]);
                }
            }
            if (!ok) give_up();
            // every MMA issued by this thread completes before TMEM is released
            umma::commit(mdone);
            (void)mbar_wait_bounded(mdone, 0u, WAIT_LIMIT);
        }
        __syncwarp();
    } else if (warp == C::LOAD_WARP) {
        // ---- weights: one bulk copy per step into the buffer of the step's parity
        if (lane == 0) {
            uint32_t issued[2] = {0u, 0u};
            int64_t gs = 0;
            bool ok = true;
            for (int64_t k = 0; k < my_groups && ok; ++k) {
                const bool dens = dens_of(blockIdx.x + k * gridDim.x);
                for (int step = 0; step < f.K; ++step, ++gs) {
                    const int b = (int)(gs & 1);
                    const int l = dens ? f.K - 1 - step : step;
                    if (gs >= 2 && !mbar_wait_bounded(&wempty[b], (uint32_t)((gs >> 1) - 1) & 1u, WAIT_LIMIT)) {
                        ok = false;
                        break;
                    }
                    if (*fail) {
                        ok = false;
                        break;
                    }
                    fence_proxy_async_smem();
                    mbar_expect_tx(&wfull[b], umma::LAYER);
                    bulk_g2s(smem + C::S_W + b * umma::LAYER, wglob + (size_t)l * umma::LAYER, umma::LAYER,
                             &wfull[b]);
                    ++issued[b];
                }
            }
            if (!ok) give_up();
            // copies in flight land before the CTA's shared memory goes away
            for (int b = 0; b < 2; ++b)
                if (issued[b]) (void)mbar_wait_bounded(&wfull[b], (issued[b] - 1u) & 1u, WAIT_LIMIT);
        }
        __syncwarp();
    }
    umma::fence_before();
    __syncthreads();
    umma::fence_after();
    if (warp == C::MMA_WARP)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(C::TMEM_COLS)
                     : "memory");
}

}  // namespace

struct fd_flow {
    int device;
    int D, K, Hd;
    int64_t n_params;
    std::vector<LayerIdx> idx;
    LayerIdx *d_idx = nullptr;
    float *d_blob = nullptr, *d_m = nullptr, *d_v = nullptr, *d_grad = nullptr, *d_gpad = nullptr;
    unsigned char *d_wpack = nullptr;
    unsigned char *d_wumma = nullptr;   // weights in the tcgen05 operand layout
    int tensor_path = 2;                // sampling / density: 0 mma.sync, 1 tcgen05 (tile pairs), 2 tcgen05 warp-specialised
    double *d_wsum = nullptr;
    float *d_loss = nullptr;
    float *d_vbuf = nullptr, *d_gbuf = nullptr;
    int64_t scratch_n = 0;
    int64_t step = 0;
};

namespace {
FlowDims dims_of(const fd_flow *f) { return FlowDims{f->D, f->K, (f->D + 1) / 2}; }

fd_status repack(fd_flow *f, cudaStream_t s) {
    pack_weights_kernel<<<dim3(32, f->K), 256, 0, s>>>(f->d_blob, f->d_idx, f->K, f->d_wpack);
    FD_CHECK_CUDA(cudaGetLastError());
    pack_umma_kernel<<<dim3(32, f->K), 256, 0, s>>>(f->d_blob, f->d_idx, f->K, f->d_wumma);
    FD_CHECK_CUDA(cudaGetLastError());
    return FD_OK;
}

int pass_smem() { return LAYER_BYTES + BLOCK * YS * 4 + BLOCK * 4 + 16; }

fd_status ensure_scratch(fd_flow *f, int64_t n) {
    if (f->scratch_n >= n) return FD_OK;
    cudaFree(f->d_vbuf);
    cudaFree(f->d_gbuf);
    f->d_vbuf = f->d_gbuf = nullptr;
    f->scratch_n = 0;
    FD_CHECK_CUDA(cudaMalloc(&f->d_vbuf, (size_t)f->D * n * 4));
    FD_CHECK_CUDA(cudaMalloc(&f->d_gbuf, (size_t)f->D * n * 4));
    f->scratch_n = n;
    return FD_OK;
}

int grid_for(int64_t units, int per_sm_ctas) {
    int dev = 0, n_sm = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    const int64_t g = std::min<int64_t>(units, (int64_t)n_sm * per_sm_ctas);
    return (int)std::max<int64_t>(g, 1);
}

template <class C>
fd_status launch_ws(const fd_flow *f, int mode, int64_t n, uint64_t seed, uint64_t iter, int32_t inst,
                    const float *xin, float *xout, float *wout, int64_t n_flow, float alpha, cudaStream_t st) {
    FD_CHECK_CUDA(cudaFuncSetAttribute(flow_ws_kernel<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM));
    flow_ws_kernel<C><<<grid_for((n + C::GROUP - 1) / C::GROUP, 1), C::THREADS, C::SMEM, st>>>(
        f->d_wumma, dims_of(f), mode, n, (uint32_t)seed, (uint32_t)(seed >> 32), (uint32_t)iter, (uint32_t)inst, xin,
        xout, wout, fd::device_status_word(), n_flow, alpha);
    FD_CHECK_CUDA(cudaGetLastError());
    return FD_OK;
}

// sampling (mode 0, flow share [0, n_flow), weights 1 / ((1 - alpha) q + alpha)) or density (mode 1)
fd_status launch_pass(const fd_flow *f, int mode, int64_t n, uint64_t seed, uint64_t iter, int32_t inst,
                      const float *xin, float *xout, float *wout, int64_t n_flow, float alpha, cudaStream_t st) {
    if (f->tensor_path == 2) {
        return launch_ws<ws::Default>(f, mode, n, seed, iter, inst, xin, xout, wout, n_flow, alpha, st);
    } else if (f->tensor_path == 1) {
        FD_CHECK_CUDA(cudaFuncSetAttribute(flow_umma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           umma::SMEM));
        flow_umma_kernel<<<grid_for((n + umma::BLOCK_U - 1) / umma::BLOCK_U, 1), umma::THREADS, umma::SMEM, st>>>(
            f->d_wumma, dims_of(f), mode, n, (uint32_t)seed, (uint32_t)(seed >> 32), (uint32_t)iter, (uint32_t)inst,
            xin, xout, wout, fd::device_status_word(), n_flow, alpha);
    } else {
        const int sm = pass_smem();
        FD_CHECK_CUDA(cudaFuncSetAttribute(flow_pass_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
        flow_pass_kernel<<<grid_for((n + BLOCK - 1) / BLOCK, 2), 128, sm, st>>>(
            f->d_wpack, dims_of(f), mode, n, (uint32_t)seed, (uint32_t)(seed >> 32), (uint32_t)iter, (uint32_t)inst,
            xin, xout, wout, fd::device_status_word(), n_flow, alpha);
    }
    FD_CHECK_CUDA(cudaGetLastError());
    return FD_OK;
}

// loss and gradient (padded per-layer, then blob layout in d_grad) of the batch
fd_status grad_impl(fd_flow *f, const float *x, const float *w, int64_t n, cudaStream_t s) {
    fd_status st = ensure_scratch(f, n);
    if (st != FD_OK) return st;
    const FlowDims fd_ = dims_of(f);
    int *status = fd::device_status_word();
    FD_CHECK_CUDA(cudaMemsetAsync(f->d_wsum, 0, sizeof(double), s));
    FD_CHECK_CUDA(cudaMemsetAsync(f->d_loss, 0, sizeof(float), s));
    FD_CHECK_CUDA(cudaMemsetAsync(f->d_gpad, 0, (size_t)f->K * GRAD_LAYER * 4, s));
    sum_weights_kernel<<<256, 256, 0, s>>>(w, n, f->d_wsum);
    FD_CHECK_CUDA(cudaGetLastError());
    const int sm1 = pass_smem();
    FD_CHECK_CUDA(cudaFuncSetAttribute(flow_inverse_train_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, sm1));
    flow_inverse_train_kernel<<<grid_for((n + BLOCK - 1) / BLOCK, 2), 128, sm1, s>>>(
        f->d_wpack, fd_, n, x, w, f->d_wsum, f->d_vbuf, f->d_gbuf, f->d_loss, status);
    FD_CHECK_CUDA(cudaGetLastError());
    const int sm2 = BwdSmem::TOTAL;
    FD_CHECK_CUDA(cudaFuncSetAttribute(flow_backward_layer_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, sm2));
    for (int l = 0; l < f->K; ++l) {
        flow_backward_layer_kernel<<<grid_for((n + 63) / 64, 1), 128, sm2, s>>>(
            f->d_wpack, fd_, l, n, w, f->d_wsum, f->d_vbuf, f->d_gbuf, f->d_gpad + (size_t)l * GRAD_LAYER, status);
        FD_CHECK_CUDA(cudaGetLastError());
    }
    unpack_grad_kernel<<<dim3(16, f->K), 256, 0, s>>>(f->d_gpad, f->d_idx, f->K, f->d_grad);
    FD_CHECK_CUDA(cudaGetLastError());
    return FD_OK;
}
}  // namespace

extern "C" fd_status fd_flow_create(int32_t dim, int32_t n_layers, int32_t hidden, uint64_t seed, fd_flow **out) {
    FD_REQUIRE(out, "out is required");
    *out = nullptr;
    FD_REQUIRE(dim >= 2 && dim <= YS, "dim must be in [2, 24] (coordinate rows of the flow kernels)");
    FD_REQUIRE(n_layers >= 1 && n_layers <= 64, "n_layers must be in [1, 64]");
    FD_REQUIRE(hidden == H, "hidden must be 128 (the tensor-core kernels' tiling)");
    fd_flow *f = new fd_flow();
    f->D = dim;
    f->K = n_layers;
    f->Hd = hidden;
    FD_CHECK_CUDA(cudaGetDevice(&f->device));
    const int h = (dim + 1) / 2;
    int64_t off = 0;
    for (int l = 0; l < n_layers; ++l) {
        LayerIdx L;
        L.a = (l % 2 == 0) ? h : dim - h;
        L.b = dim - L.a;
        L.off = off;
        off += (int64_t)H * L.a + H + (int64_t)H * H + H + 2LL * L.b * H + 2 * L.b;
        f->idx.push_back(L);
        if (L.a > 16 || L.b > 16) {
            delete f;
            return fd::set_error(FD_ENOTSUP, "coupling halves larger than 16 coordinates");
        }
    }
    f->n_params = off;
    // initial weights: uniform(+-1/sqrt(fan_in)) for W1, W2 and zero output layer (identity flow)
    std::vector<float> blob(off, 0.f);
    uint64_t st = seed * 0x9E3779B97F4A7C15ull + 1;
    auto rnd = [&]() {
        st ^= st << 13;
        st ^= st >> 7;
        st ^= st << 17;
        return (double)(st >> 11) * (1.0 / 9007199254740992.0);
    };
    for (int l = 0; l < n_layers; ++l) {
        const LayerIdx &L = f->idx[l];
        float *W1 = blob.data() + L.off;
        float *W2 = W1 + H * L.a + H;
        for (int k = 0; k < H * L.a; ++k) W1[k] = (float)((2 * rnd() - 1) / std::sqrt((double)L.a));
        for (int k = 0; k < H * H; ++k) W2[k] = (float)((2 * rnd() - 1) / std::sqrt((double)H));
    }
    cudaError_t e = cudaSuccess;
    auto al = [&](void **p, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(p, bytes);
        if (e == cudaSuccess) e = cudaMemset(*p, 0, bytes);
    };
    al((void **)&f->d_blob, off * 4);
    al((void **)&f->d_m, off * 4);
    al((void **)&f->d_v, off * 4);
    al((void **)&f->d_grad, off * 4);
    al((void **)&f->d_gpad, (size_t)n_layers * GRAD_LAYER * 4);
    al((void **)&f->d_wpack, (size_t)n_layers * LAYER_BYTES);
    al((void **)&f->d_wumma, (size_t)n_layers * umma::LAYER);
    al((void **)&f->d_idx, n_layers * sizeof(LayerIdx));
    al((void **)&f->d_wsum, sizeof(double));
    al((void **)&f->d_loss, sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpy(f->d_idx, f->idx.data(), n_layers * sizeof(LayerIdx), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(f->d_blob, blob.data(), off * 4, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        fd_flow_free(f);
        return fd::cuda_error(e, "fd_flow_create");
    }
    fd_status s2 = repack(f, 0);
    if (s2 == FD_OK) {
        cudaError_t e2 = cudaDeviceSynchronize();
        if (e2 != cudaSuccess) s2 = fd::cuda_error(e2, "fd_flow_create");
    }
    if (s2 != FD_OK) {
        fd_flow_free(f);
        return s2;
    }
    *out = f;
    return FD_OK;
}

extern "C" void fd_flow_free(fd_flow *f) {
    if (!f) return;
    cudaFree(f->d_blob);
    cudaFree(f->d_m);
    cudaFree(f->d_v);
    cudaFree(f->d_grad);
    cudaFree(f->d_gpad);
    cudaFree(f->d_wpack);
    cudaFree(f->d_wumma);
    cudaFree(f->d_idx);
    cudaFree(f->d_wsum);
    cudaFree(f->d_loss);
    cudaFree(f->d_vbuf);
    cudaFree(f->d_gbuf);
    delete f;
}

extern "C" int64_t fd_flow_param_count(const fd_flow *f) { return f ? f->n_params : 0; }

extern "C" fd_status fd_flow_set_params(fd_flow *f, const float *blob, int64_t n) {
    FD_REQUIRE(f && blob, "flow and blob are required");
    FD_REQUIRE(n == f->n_params, "blob size differs from fd_flow_param_count");
    for (int64_t k = 0; k < n; ++k) FD_REQUIRE(std::isfinite(blob[k]), "non-finite parameter");
    FD_CHECK_CUDA(cudaDeviceSynchronize());
    FD_CHECK_CUDA(cudaMemcpy(f->d_blob, blob, n * 4, cudaMemcpyHostToDevice));
    FD_CHECK_CUDA(cudaMemset(f->d_m, 0, n * 4));
    FD_CHECK_CUDA(cudaMemset(f->d_v, 0, n * 4));
    f->step = 0;
    fd_status st = repack(f, 0);
    if (st != FD_OK) return st;
    FD_CHECK_CUDA(cudaDeviceSynchronize());
    return FD_OK;
}

extern "C" fd_status fd_flow_get_params(const fd_flow *f, float *blob, int64_t n) {
    FD_REQUIRE(f && blob, "flow and blob are required");
    FD_REQUIRE(n == f->n_params, "blob size differs from fd_flow_param_count");
    FD_CHECK_CUDA(cudaDeviceSynchronize());
    FD_CHECK_CUDA(cudaMemcpy(blob, f->d_blob, n * 4, cudaMemcpyDeviceToHost));
    return FD_OK;
}

extern "C" fd_status fd_flow_sample(const fd_flow *f, uint64_t seed, uint64_t iter, int32_t inst, int64_t n,
                                    float *x, float *w, void *stream) {
    FD_REQUIRE(f && x && w, "flow, x and w are required");
    FD_REQUIRE(n > 0 && n <= (int64_t(1) << 34), "n out of range");
    FD_REQUIRE(inst >= 0 && inst < (1 << 24), "instance index out of range");
    return launch_pass(f, 0, n, seed, iter, inst, nullptr, x, w, n, 0.0f, (cudaStream_t)stream);
}

extern "C" fd_status fd_flow_sample_defensive(const fd_flow *f, uint64_t seed, uint64_t iter, int32_t inst,
                                              int64_t n, double alpha, float *x, float *w, double *alpha_used,
                                              void *stream) {
    FD_REQUIRE(f && x && w, "flow, x and w are required");
    FD_REQUIRE(n > 0 && n <= (int64_t(1) << 34), "n out of range");
    FD_REQUIRE(inst >= 0 && inst < (1 << 24), "instance index out of range");
    FD_REQUIRE(alpha >= 0.0 && alpha <= 0.5, "alpha must be in [0, 0.5]");
    // the flow share ends on a block boundary of both sampling kernels, so every block is of one kind
    constexpr int64_t UNIT = umma::BLOCK_U;
    static_assert(UNIT % BLOCK == 0 && UNIT % ws::Default::GROUP == 0,
                  "the flow share ends on every kernel's block boundary");
    const int64_t n_flow = std::min(n, (n - (int64_t)(alpha * (double)n) + UNIT - 1) / UNIT * UNIT);
    const int64_t n_u = n - n_flow;
    const float a = (float)((double)n_u / (double)n);
    if (alpha_used) *alpha_used = (double)n_u / (double)n;
    return launch_pass(f, 0, n, seed, iter, inst, nullptr, x, w, n_flow, a, (cudaStream_t)stream);
}

extern "C" fd_status fd_flow_log_density(const fd_flow *f, const float *x, int64_t n, float *logq, void *stream) {
    FD_REQUIRE(f && x && logq, "flow, x and logq are required");
    FD_REQUIRE(n > 0 && n <= (int64_t(1) << 34), "n out of range");
    return launch_pass(f, 1, n, 0, 0, 0, x, nullptr, logq, n, 0.0f, (cudaStream_t)stream);
}

extern "C" fd_status fd_flow_set_tensor_path(fd_flow *f, int32_t path) {
    FD_REQUIRE(f, "null flow");
    FD_REQUIRE(path >= 0 && path <= 2, "path must be 0 (mma.sync), 1 (tcgen05) or 2 (tcgen05, warp-specialised)");
    f->tensor_path = path;
    return FD_OK;
}

extern "C" fd_status fd_flow_grad(fd_flow *f, const float *x, const float *w, int64_t n, float *loss, float *grad,
                                  void *stream) {
    FD_REQUIRE(f && x && w && loss && grad, "flow, x, w, loss and grad are required");
    FD_REQUIRE(n > 0 && n <= (int64_t(1) << 30), "n out of range");
    cudaStream_t s = (cudaStream_t)stream;
    fd_status st = grad_impl(f, x, w, n, s);
    if (st != FD_OK) return st;
    FD_CHECK_CUDA(cudaMemcpyAsync(loss, f->d_loss, sizeof(float), cudaMemcpyDeviceToDevice, s));
    FD_CHECK_CUDA(cudaMemcpyAsync(grad, f->d_grad, f->n_params * 4, cudaMemcpyDeviceToDevice, s));
    return FD_OK;
}

extern "C" fd_status fd_flow_train(fd_flow *f, const float *x, const float *w, int64_t n, int32_t steps, float lr,
                                   float *loss_out, void *stream) {
    FD_REQUIRE(f && x && w, "flow, x and w are required");
    FD_REQUIRE(n > 0 && n <= (int64_t(1) << 30), "n out of range");
    FD_REQUIRE(steps >= 1 && lr > 0.f && std::isfinite(lr), "steps >= 1 and a positive learning rate are required");
    cudaStream_t s = (cudaStream_t)stream;
    float *d_losses = nullptr;
    if (loss_out) FD_CHECK_CUDA(cudaMalloc(&d_losses, steps * sizeof(float)));
    for (int k = 0; k < steps; ++k) {
        fd_status st = grad_impl(f, x, w, n, s);
        if (st != FD_OK) {
            cudaFree(d_losses);
            return st;
        }
        if (d_losses) FD_CHECK_CUDA(cudaMemcpyAsync(d_losses + k, f->d_loss, 4, cudaMemcpyDeviceToDevice, s));
        f->step += 1;
        const float b1t = (float)std::pow(0.9, (double)f->step), b2t = (float)std::pow(0.999, (double)f->step);
        adam_kernel<<<(unsigned)((f->n_params + 255) / 256), 256, 0, s>>>(f->d_blob, f->d_grad, f->d_m, f->d_v,
                                                                          f->n_params, lr, b1t, b2t);
        FD_CHECK_CUDA(cudaGetLastError());
        st = repack(f, s);
        if (st != FD_OK) {
            cudaFree(d_losses);
            return st;
        }
    }
    if (loss_out) {
        FD_CHECK_CUDA(cudaMemcpyAsync(loss_out, d_losses, steps * sizeof(float), cudaMemcpyDeviceToHost, s));
        FD_CHECK_CUDA(cudaStreamSynchronize(s));
        cudaFree(d_losses);
    }
    return FD_OK;
}
