// Neural spline flow, sampling and density (App. A): x = T(z) with z uniform
// on the unit hypercube and T a stack of rational-quadratic coupling layers
// (Durkan et al., 2019: K = 8 bins, knots from softmax widths and heights,
// softplus derivatives at the internal knots, derivative 1 at both ends), the
// spline parameters of every transformed coordinate produced by a residual
// conditioner (linear to width 32, two residual blocks of two 32x32 layers
// with ReLU, linear to 3K - 1 outputs per coordinate) from the unchanged
// coordinates.  Coupling layers alternate which half stays unchanged (layer
// 2i keeps the first floor(D/2) coordinates).  log q(x) = -sum of the
// transformed coordinates' log derivatives.
//
// One thread per sample: its D coordinates and the conditioner's hidden
// vector live in registers; the layer's weights (53 KB at D = 19) are staged
// in shared memory once per layer and block; a transformed coordinate's 23
// spline parameters are computed just before its spline, so they never need
// more than 23 registers.  FP32 arithmetic with IEEE exp/log (the parameters
// pass through softmax and softplus).
#include <cuda_bf16.h>

#include "fd_internal.cuh"
#include "fd_nsf_math.cuh"

#include <algorithm>
#include <cmath>
#include <vector>

namespace {

using namespace nsf;

struct NsfArgs {
    const float *params;      // all layers, in order
    const float *z;           // [dim][ldz] or null: Philox stream
    float *x;                 // [dim][ldx]
    float *logq;              // [n]: log q(x), or with inv_q the importance weight 1 / q(x)
    int64_t n, ldz, ldx;
    int inv_q;
    int dim, n_layers;
    uint32_t seed_lo, seed_hi, iter, inst;
};

// INV = false: z -> x = T(z); INV = true: x -> z = T^-1(x) (the layers in
// reverse order).  Both return log q(x) = -sum of the log derivatives.
template <bool INV>
__global__ void __launch_bounds__(128) nsf_kernel(const NsfArgs a) {
    extern __shared__ __align__(16) float wsm[];
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = i < a.n;
    const int D = a.dim, half = D / 2;
    float v[kMaxDim];
    if (a.z) {
#pragma unroll
        for (int j = 0; j < kMaxDim; ++j) v[j] = (j < D && valid) ? a.z[(int64_t)j * a.ldz + i] : 0.5f;
    } else {
        // the sample stream: counter (i_lo, i_hi, iter, inst << 8 | block), 4 words a block
#pragma unroll
        for (int b = 0; b < kMaxDim / 4; ++b) {
            if (4 * b >= D) break;
            const u32x4 r = philox4x32_10(u32x4{(uint32_t)i, (uint32_t)((uint64_t)i >> 32), a.iter, (a.inst << 8) | (uint32_t)b},
                                          a.seed_lo, a.seed_hi);
            const uint32_t ws[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (4 * b + q < kMaxDim) v[4 * b + q] = word_to_uniform(ws[q]);
        }
    }
    float logq = 0.0f;
    for (int step = 0; step < a.n_layers; ++step) {
        const int layer = INV ? a.n_layers - 1 - step : step;
        const float *lp = a.params + layer_offset(layer, D);
        const int keep0 = layer % 2 == 0 ? 0 : half, n_keep = layer % 2 == 0 ? half : D - half;
        const int move0 = layer % 2 == 0 ? half : 0, n_move = D - n_keep;
        const int64_t head = head_floats(n_keep);
        const int row = n_move * kParamsPerDim;                    // W1 row length in global memory
        __syncthreads();                                            // the previous layer's weights are consumed
        for (int64_t k = threadIdx.x; k < head; k += blockDim.x) wsm[k] = __ldg(lp + k);
        for (int64_t k = threadIdx.x; k < (int64_t)(kHidden + 1) * n_move * kPad; k += blockDim.x) {
            // padded index k = (r n_move + m) 24 + q; r = 32 is b1
            const int q = (int)(k % kPad);
            const int64_t rm = k / kPad;
            const int r = (int)(rm / n_move), m = (int)(rm % n_move);
            wsm[head + k] = q < kParamsPerDim ? __ldg(lp + head + (int64_t)r * row + m * kParamsPerDim + q) : 0.0f;
        }
        __syncthreads();
        const float *W0 = wsm, *b0 = W0 + n_keep * kHidden, *blk = b0 + kHidden;
        const float *W1 = wsm + head, *b1 = W1 + (int64_t)kHidden * n_move * kPad;
        float hdn[kHidden];
#pragma unroll
        for (int c = 0; c < kHidden; ++c) hdn[c] = b0[c];
        for (int r = 0; r < n_keep; ++r) {
            float xv = 0.0f;
#pragma unroll
            for (int j = 0; j < kMaxDim; ++j)
                if (j == keep0 + r) xv = v[j];
#pragma unroll
            for (int c4 = 0; c4 < kHidden / 4; ++c4) {
                const float4 w = reinterpret_cast<const float4 *>(W0 + r * kHidden)[c4];
                hdn[4 * c4] = fmaf(xv, w.x, hdn[4 * c4]);
                hdn[4 * c4 + 1] = fmaf(xv, w.y, hdn[4 * c4 + 1]);
                hdn[4 * c4 + 2] = fmaf(xv, w.z, hdn[4 * c4 + 2]);
                hdn[4 * c4 + 3] = fmaf(xv, w.w, hdn[4 * c4 + 3]);
            }
        }
#pragma unroll 1
        for (int bk = 0; bk < 2; ++bk) {
            const float *Wa = blk + bk * 2 * (kHidden * kHidden + kHidden), *ba = Wa + kHidden * kHidden;
            const float *Wb = ba + kHidden, *bb = Wb + kHidden * kHidden;
            float t[kHidden];
#pragma unroll
            for (int c = 0; c < kHidden; ++c) t[c] = ba[c];
#pragma unroll
            for (int r = 0; r < kHidden; ++r) {
                const float hr = fmaxf(hdn[r], 0.0f);
#pragma unroll
                for (int c4 = 0; c4 < kHidden / 4; ++c4) {
                    const float4 w = reinterpret_cast<const float4 *>(Wa + r * kHidden)[c4];
                    t[4 * c4] = fmaf(hr, w.x, t[4 * c4]);
                    t[4 * c4 + 1] = fmaf(hr, w.y, t[4 * c4 + 1]);
                    t[4 * c4 + 2] = fmaf(hr, w.z, t[4 * c4 + 2]);
                    t[4 * c4 + 3] = fmaf(hr, w.w, t[4 * c4 + 3]);
                }
            }
            float t2[kHidden];
#pragma unroll
            for (int c = 0; c < kHidden; ++c) t2[c] = bb[c];
#pragma unroll
            for (int r = 0; r < kHidden; ++r) {
                const float tr = fmaxf(t[r], 0.0f);
#pragma unroll
                for (int c4 = 0; c4 < kHidden / 4; ++c4) {
                    const float4 w = reinterpret_cast<const float4 *>(Wb + r * kHidden)[c4];
                    t2[4 * c4] = fmaf(tr, w.x, t2[4 * c4]);
                    t2[4 * c4 + 1] = fmaf(tr, w.y, t2[4 * c4 + 1]);
                    t2[4 * c4 + 2] = fmaf(tr, w.z, t2[4 * c4 + 2]);
                    t2[4 * c4 + 3] = fmaf(tr, w.w, t2[4 * c4 + 3]);
                }
            }
#pragma unroll
            for (int c = 0; c < kHidden; ++c) hdn[c] += t2[c];
        }
        for (int m = 0; m < n_move; ++m) {
            float p[kPad];
#pragma unroll
            for (int q4 = 0; q4 < kPad / 4; ++q4) {
                const float4 b = reinterpret_cast<const float4 *>(b1 + m * kPad)[q4];
                p[4 * q4] = b.x;
                p[4 * q4 + 1] = b.y;
                p[4 * q4 + 2] = b.z;
                p[4 * q4 + 3] = b.w;
            }
#pragma unroll
            for (int r = 0; r < kHidden; ++r) {
                const float4 *w4 = reinterpret_cast<const float4 *>(W1 + ((int64_t)r * n_move + m) * kPad);
#pragma unroll
                for (int q4 = 0; q4 < kPad / 4; ++q4) {
                    const float4 w = w4[q4];
                    p[4 * q4] = fmaf(hdn[r], w.x, p[4 * q4]);
                    p[4 * q4 + 1] = fmaf(hdn[r], w.y, p[4 * q4 + 1]);
                    p[4 * q4 + 2] = fmaf(hdn[r], w.z, p[4 * q4 + 2]);
                    if (4 * q4 + 3 < kParamsPerDim) p[4 * q4 + 3] = fmaf(hdn[r], w.w, p[4 * q4 + 3]);
                }
            }
            float u = 0.0f;
#pragma unroll
            for (int j = 0; j < kMaxDim; ++j)
                if (j == move0 + m) u = v[j];
            float y, logd;
            if (INV)
                rq_spline_inverse(p, fminf(fmaxf(u, 0.0f), 1.0f), y, logd);
            else
                rq_spline(p, fminf(fmaxf(u, 0.0f), 1.0f), y, logd);
#pragma unroll
            for (int j = 0; j < kMaxDim; ++j)
                if (j == move0 + m) v[j] = y;
            logq -= logd;
        }
    }
    if (!valid) return;
#pragma unroll
    for (int j = 0; j < kMaxDim; ++j)
        if (j < D) a.x[(int64_t)j * a.ldx + i] = v[j];
    a.logq[i] = a.inv_q ? expf(-logq) : logq;
}


// ---- sampling and density with the conditioner on the tensor cores ----------------
// The conditioner's GEMMs as warp-level mma.sync m16n8k16 tiles: BF16 weights
// and GEMM inputs (the kept coordinates, relu(h), relu(t), h2), FP32
// accumulation and an FP32 residual stream (the BF16 contract of the affine
// flow's sampler).  A warp takes 32 samples (two 16-row tiles); a CTA of four
// warps takes ROUNDS tiles of 128 samples per staging of a layer's weights.
// Per layer: h = W0 x_keep + b0 and the two residual blocks stay in
// registers (accumulators become the next GEMM's A fragments); the 24
// outputs of every moved coordinate (23 spline parameters and a zero) go
// through a per-warp scratch to the sample's own thread, which evaluates the
// spline in FP32 as in nsf_kernel.  A sample's coordinates live in a shared
// memory row.
namespace nsf_tc {
constexpr int ROUNDS = 2;
constexpr int WARPS = 4, THREADS = 32 * WARPS, BLOCK = THREADS * ROUNDS;
constexpr int LD16 = 24, LD32 = 40;     // BF16 row pitches of the staged W^T (conflict-free fragment loads)
constexpr int VROW = 25, PROW = 25;     // floats per coordinate row and per parameter row (odd)
constexpr int MAXMOVE = kMaxDim / 2;    // at most 12 moved coordinates per layer
// staged layer, BF16 part: W0^T [32][LD16], Wa^T, Wb^T of both blocks [32][LD32], W1^T [n_move * 24][LD32]
constexpr int OFF_W0 = 0, OFF_WA = OFF_W0 + kHidden * LD16, OFF_WB = OFF_WA + 2 * kHidden * LD32;
constexpr int OFF_W1 = OFF_WB + 2 * kHidden * LD32;
constexpr int BF_ELEMS = OFF_W1 + MAXMOVE * kPad * LD32;
// FP32 part: b0 [32], ba [2][32], bb [2][32], b1 [n_move * 24]
constexpr int F_B0 = 0, F_BA = kHidden, F_BB = 3 * kHidden, F_B1 = 5 * kHidden;
constexpr int F_ELEMS = F_B1 + MAXMOVE * kPad;
constexpr size_t SMEM = (size_t)BF_ELEMS * 2 + (size_t)F_ELEMS * 4 + (size_t)BLOCK * VROW * 4 +
                        (size_t)WARPS * 32 * PROW * 4;
static_assert((BF_ELEMS * 2) % 16 == 0, "alignment of the FP32 part");

__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&v);
}
__device__ __forceinline__ uint32_t relu2(float lo, float hi) {
    uint32_t d;
    asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    return d;
}
__device__ __forceinline__ void mma(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
// B fragment (k-tile kt, n-tile nt) of B = W (K x N) from W^T rows of pitch ld
__device__ __forceinline__ void bfrag(const __nv_bfloat16 *WT, int ld, int kt, int nt, int g, int t, uint32_t &b0,
                                      uint32_t &b1) {
    const __nv_bfloat16 *p = WT + (nt * 8 + g) * ld + kt * 16 + 2 * t;
    b0 = *reinterpret_cast<const uint32_t *>(p);
    b1 = *reinterpret_cast<const uint32_t *>(p + 8);
}
// accumulators of n-tiles (2j, 2j+1) -> the A fragment of k-tile j (ReLU or not)
template <bool RELU>
__device__ __forceinline__ void c_to_a(const float (&c0)[4], const float (&c1)[4], uint32_t (&a)[4]) {
    if (RELU) {
        a[0] = relu2(c0[0], c0[1]);
        a[1] = relu2(c0[2], c0[3]);
        a[2] = relu2(c1[0], c1[1]);
        a[3] = relu2(c1[2], c1[3]);
    } else {
        a[0] = pack2(c0[0], c0[1]);
        a[1] = pack2(c0[2], c0[3]);
        a[2] = pack2(c1[0], c1[1]);
        a[3] = pack2(c1[2], c1[3]);
    }
}

// one layer's weights, BF16 and transposed (outputs by rows), from the parameter vector
__device__ void stage(const float *lp, int n_keep, int n_move, __nv_bfloat16 *bw, float *fw) {
    const int row = n_move * kParamsPerDim;                 // W1 row length in the parameter vector
    const float *W0 = lp, *b0 = W0 + n_keep * kHidden, *blk = b0 + kHidden;
    const float *W1 = lp + head_floats(n_keep), *b1 = W1 + (int64_t)kHidden * row;
    __syncthreads();                                        // the previous layer's weights are consumed
    for (int k = threadIdx.x; k < kHidden * 16; k += THREADS) {
        const int nn = k / 16, kk = k % 16;
        bw[OFF_W0 + nn * LD16 + kk] = __float2bfloat16_rn(kk < n_keep ? W0[kk * kHidden + nn] : 0.0f);
    }
    for (int k = threadIdx.x; k < 4 * kHidden * kHidden; k += THREADS) {
        const int mat = k / (kHidden * kHidden), e = k % (kHidden * kHidden), nn = e / kHidden, kk = e % kHidden;
        const int bk = mat >> 1, second = mat & 1;         // Wa0, Wb0, Wa1, Wb1
        const float *W = blk + bk * 2 * (kHidden * kHidden + kHidden) + second * (kHidden * kHidden + kHidden);
        bw[(second ? OFF_WB : OFF_WA) + bk * kHidden * LD32 + nn * LD32 + kk] = __float2bfloat16_rn(W[kk * kHidden + nn]);
    }
    for (int k = threadIdx.x; k < n_move * kPad * kHidden; k += THREADS) {
        const int nn = k / kHidden, kk = k % kHidden, m = nn / kPad, q = nn % kPad;
        bw[OFF_W1 + nn * LD32 + kk] =
            __float2bfloat16_rn(q < kParamsPerDim ? W1[(int64_t)kk * row + m * kParamsPerDim + q] : 0.0f);
    }
    for (int k = threadIdx.x; k < kHidden; k += THREADS) {
        fw[F_B0 + k] = b0[k];
        for (int bk = 0; bk < 2; ++bk) {
            const float *Wa = blk + bk * 2 * (kHidden * kHidden + kHidden);
            fw[F_BA + bk * kHidden + k] = Wa[kHidden * kHidden + k];
            fw[F_BB + bk * kHidden + k] = Wa[2 * kHidden * kHidden + kHidden + k];
        }
    }
    for (int k = threadIdx.x; k < n_move * kPad; k += THREADS) {
        const int m = k / kPad, q = k % kPad;
        fw[F_B1 + k] = q < kParamsPerDim ? b1[m * kParamsPerDim + q] : 0.0f;
    }
    __syncthreads();
}
}  // namespace nsf_tc

template <bool INV>
__global__ void __launch_bounds__(nsf_tc::THREADS) nsf_tc_kernel(const NsfArgs a) {
    using namespace nsf_tc;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __nv_bfloat16 *bw = reinterpret_cast<__nv_bfloat16 *>(smem_raw);
    float *fw = reinterpret_cast<float *>(smem_raw + (size_t)BF_ELEMS * 2);
    float *V = fw + F_ELEMS;                                // [BLOCK][VROW] coordinates
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    float *P = V + BLOCK * VROW + warp * 32 * PROW;         // this warp's [32][PROW] spline parameters
    const int D = a.dim, half = D / 2;
    const int64_t base = (int64_t)blockIdx.x * BLOCK;
    // the coordinates of the block's samples (sample r of the block in row r)
    float logq[ROUNDS];
    for (int r = 0; r < ROUNDS; ++r) {
        const int row = r * THREADS + threadIdx.x;
        const int64_t i = base + row;
        const bool valid = i < a.n;
        float *v = V + row * VROW;
        logq[r] = 0.0f;
        if (a.z) {
            for (int j = 0; j < D; ++j) v[j] = valid ? a.z[(int64_t)j * a.ldz + i] : 0.5f;
        } else {
            for (int b = 0; 4 * b < D; ++b) {
                const u32x4 rr = philox4x32_10(u32x4{(uint32_t)i, (uint32_t)((uint64_t)i >> 32), a.iter,
                                                     (a.inst << 8) | (uint32_t)b},
                                               a.seed_lo, a.seed_hi);
                const uint32_t ws[4] = {rr.x, rr.y, rr.z, rr.w};
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (4 * b + q < D) v[4 * b + q] = word_to_uniform(ws[q]);
            }
        }
    }
    for (int step = 0; step < a.n_layers; ++step) {
        const int layer = INV ? a.n_layers - 1 - step : step;
        const int keep0 = layer % 2 == 0 ? 0 : half, n_keep = layer % 2 == 0 ? half : D - half;
        const int move0 = layer % 2 == 0 ? half : 0, n_move = D - n_keep;
        stage(a.params + layer_offset(layer, D), n_keep, n_move, bw, fw);
        for (int r = 0; r < ROUNDS; ++r) {
            const float *Vt = V + (r * THREADS + warp * 32) * VROW;   // this warp's 32 rows
            // input fragments: the kept coordinates (K = 16, zero beyond n_keep)
            uint32_t ax[2][4];
#pragma unroll
            for (int rt = 0; rt < 2; ++rt) {
                const float *r0 = Vt + (16 * rt + g) * VROW + keep0, *r1 = r0 + 8 * VROW;
                auto kv = [&](const float *rw, int k) { return k < n_keep ? rw[k] : 0.0f; };
                ax[rt][0] = pack2(kv(r0, 2 * t), kv(r0, 2 * t + 1));
                ax[rt][1] = pack2(kv(r1, 2 * t), kv(r1, 2 * t + 1));
                ax[rt][2] = pack2(kv(r0, 2 * t + 8), kv(r0, 2 * t + 9));
                ax[rt][3] = pack2(kv(r1, 2 * t + 8), kv(r1, 2 * t + 9));
            }
            // h = W0 x + b0
            float h[2][4][4];
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) {
                const float u0 = fw[F_B0 + nt * 8 + 2 * t], u1 = fw[F_B0 + nt * 8 + 2 * t + 1];
                uint32_t b0, b1;
                bfrag(bw + OFF_W0, LD16, 0, nt, g, t, b0, b1);
#pragma unroll
                for (int rt = 0; rt < 2; ++rt) {
                    h[rt][nt][0] = u0;
                    h[rt][nt][1] = u1;
                    h[rt][nt][2] = u0;
                    h[rt][nt][3] = u1;
                    mma(h[rt][nt], ax[rt], b0, b1);
                }
            }
            // two residual blocks: h += Wb relu(Wa relu(h) + ba) + bb
#pragma unroll
            for (int bk = 0; bk < 2; ++bk) {
                const __nv_bfloat16 *WaT = bw + OFF_WA + bk * kHidden * LD32, *WbT = bw + OFF_WB + bk * kHidden * LD32;
                uint32_t ah[2][2][4];
#pragma unroll
                for (int rt = 0; rt < 2; ++rt)
#pragma unroll
                    for (int kt = 0; kt < 2; ++kt) c_to_a<true>(h[rt][2 * kt], h[rt][2 * kt + 1], ah[rt][kt]);
                float tt[2][4][4];
#pragma unroll
                for (int nt = 0; nt < 4; ++nt) {
                    const float u0 = fw[F_BA + bk * kHidden + nt * 8 + 2 * t];
                    const float u1 = fw[F_BA + bk * kHidden + nt * 8 + 2 * t + 1];
#pragma unroll
                    for (int rt = 0; rt < 2; ++rt) {
                        tt[rt][nt][0] = u0;
                        tt[rt][nt][1] = u1;
                        tt[rt][nt][2] = u0;
                        tt[rt][nt][3] = u1;
                    }
#pragma unroll
                    for (int kt = 0; kt < 2; ++kt) {
                        uint32_t b0, b1;
                        bfrag(WaT, LD32, kt, nt, g, t, b0, b1);
#pragma unroll
                        for (int rt = 0; rt < 2; ++rt) mma(tt[rt][nt], ah[rt][kt], b0, b1);
                    }
                }
                uint32_t at[2][2][4];
#pragma unroll
                for (int rt = 0; rt < 2; ++rt)
#pragma unroll
                    for (int kt = 0; kt < 2; ++kt) c_to_a<true>(tt[rt][2 * kt], tt[rt][2 * kt + 1], at[rt][kt]);
#pragma unroll
                for (int nt = 0; nt < 4; ++nt) {
                    const float u0 = fw[F_BB + bk * kHidden + nt * 8 + 2 * t];
                    const float u1 = fw[F_BB + bk * kHidden + nt * 8 + 2 * t + 1];
#pragma unroll
                    for (int rt = 0; rt < 2; ++rt) {
                        h[rt][nt][0] += u0;
                        h[rt][nt][1] += u1;
                        h[rt][nt][2] += u0;
                        h[rt][nt][3] += u1;
                    }
#pragma unroll
                    for (int kt = 0; kt < 2; ++kt) {
                        uint32_t b0, b1;
                        bfrag(WbT, LD32, kt, nt, g, t, b0, b1);
#pragma unroll
                        for (int rt = 0; rt < 2; ++rt) mma(h[rt][nt], at[rt][kt], b0, b1);
                    }
                }
            }
            uint32_t a2[2][2][4];
#pragma unroll
            for (int rt = 0; rt < 2; ++rt)
#pragma unroll
                for (int kt = 0; kt < 2; ++kt) c_to_a<false>(h[rt][2 * kt], h[rt][2 * kt + 1], a2[rt][kt]);
            // every moved coordinate: its 24 outputs through the warp's scratch to its sample's thread
            float *vme = V + (r * THREADS + threadIdx.x) * VROW;
            for (int m = 0; m < n_move; ++m) {
#pragma unroll
                for (int nt = 0; nt < 3; ++nt) {
                    const int c0 = m * kPad + nt * 8 + 2 * t;
                    const float u0 = fw[F_B1 + c0], u1 = fw[F_B1 + c0 + 1];
                    float pc[2][4] = {{u0, u1, u0, u1}, {u0, u1, u0, u1}};
#pragma unroll
                    for (int kt = 0; kt < 2; ++kt) {
                        uint32_t b0, b1;
                        bfrag(bw + OFF_W1 + m * kPad * LD32, LD32, kt, nt, g, t, b0, b1);
#pragma unroll
                        for (int rt = 0; rt < 2; ++rt) mma(pc[rt], a2[rt][kt], b0, b1);
                    }
#pragma unroll
                    for (int rt = 0; rt < 2; ++rt) {
                        float *p0 = P + (16 * rt + g) * PROW + nt * 8 + 2 * t, *p1 = p0 + 8 * PROW;
                        p0[0] = pc[rt][0];
                        p0[1] = pc[rt][1];
                        p1[0] = pc[rt][2];
                        p1[1] = pc[rt][3];
                    }
                }
                __syncwarp();
                float p[kPad];
#pragma unroll
                for (int q = 0; q < kPad; ++q) p[q] = P[lane * PROW + q];
                __syncwarp();                                   // the scratch is free for the next coordinate
                float y, logd;
                const float u = fminf(fmaxf(vme[move0 + m], 0.0f), 1.0f);
                if (INV)
                    rq_spline_inverse(p, u, y, logd);
                else
                    rq_spline(p, u, y, logd);
                vme[move0 + m] = y;
                logq[r] -= logd;
            }
            __syncwarp();                                       // coordinates written before the next layer reads them
        }
    }
    for (int r = 0; r < ROUNDS; ++r) {
        const int row = r * THREADS + threadIdx.x;
        const int64_t i = base + row;
        if (i >= a.n) continue;
        const float *v = V + row * VROW;
        for (int j = 0; j < D; ++j) a.x[(int64_t)j * a.ldx + i] = v[j];
        a.logq[i] = a.inv_q ? expf(-logq[r]) : logq[r];
    }
}

// ---- gradient of the forward-KL loss (App. A) ------------------------------
// loss = -sum_i w_i log q(x_i) / sum_i w_i over given points x_i and weights
// w_i, and its gradient in every parameter by reverse mode through the
// inverse pass.  One thread per sample: the inverse pass (layers L-1 .. 0)
// keeps each layer's input in local memory; the backward sweep then walks the
// layers in the flow's order (0 .. L-1), recomputing each conditioner from
// the kept input (layer_backward).  A parameter's gradient is summed over the
// warp's samples through shared memory and added to global memory once per
// warp (WarpAtomicAcc).

constexpr int kGradMaxLayers = 16;
constexpr int kNsfMaxTrainSteps = 4096;      // losses kept per fd_nsf_train call

// The warp's accumulator: a rank-one update G[r][q] += a[r] b[q] summed over
// the warp's 32 samples is a small matrix product, computed by writing the
// lanes' a and b rows to the warp's shared-memory scratch (rows of 33
// floats: conflict-free) and letting lane r sum row r of G over the samples
// (b read as broadcasts); one atomic per entry and warp.  About 30
// instructions per 23 entries against 11 per entry for a per-entry warp
// reduction.
constexpr int kAccRow = 33;
struct WarpAtomicAcc {
    float *g;                                 // the layer's slice of the gradient
    float *s;                                 // this warp's scratch: [32][kAccRow] a rows, then b rows
};

template <int NA, int NB>
__device__ __forceinline__ void acc_outer(WarpAtomicAcc &acc, int64_t off, int64_t stride, const float (&a)[NA],
                                          int na, const float (&b)[NB], int nb) {
    const int lane = threadIdx.x & 31;
    float *A = acc.s, *B = acc.s + 32 * kAccRow;
    __syncwarp();                                            // the scratch's previous use is over
#pragma unroll
    for (int r = 0; r < NA; ++r)
        if (r < na) A[lane * kAccRow + r] = a[r];
#pragma unroll
    for (int q = 0; q < NB; ++q)
        if (q < nb) B[lane * kAccRow + q] = b[q];
    __syncwarp();
    if (lane < na) {
        float sum[NB];
#pragma unroll
        for (int q = 0; q < NB; ++q) sum[q] = 0.0f;
        for (int smp = 0; smp < 32; ++smp) {
            const float ar = A[smp * kAccRow + lane];
#pragma unroll
            for (int q = 0; q < NB; ++q) sum[q] = fmaf(ar, B[smp * kAccRow + q], sum[q]);
        }
#pragma unroll
        for (int q = 0; q < NB; ++q)
            if (q < nb && sum[q] != 0.0f) atomicAdd(acc.g + off + lane * stride + q, sum[q]);
    }
}

template <int NB>
__device__ __forceinline__ void acc_vec(WarpAtomicAcc &acc, int64_t off, const float (&b)[NB], int nb) {
    const int lane = threadIdx.x & 31;
    float *B = acc.s + 32 * kAccRow;
    __syncwarp();
#pragma unroll
    for (int q = 0; q < NB; ++q)
        if (q < nb) B[lane * kAccRow + q] = b[q];
    __syncwarp();
    if (lane < nb) {
        float sum = 0.0f;
        for (int smp = 0; smp < 32; ++smp) sum += B[smp * kAccRow + lane];
        if (sum != 0.0f) atomicAdd(acc.g + off + lane, sum);
    }
}

struct NsfGradArgs {
    const float *params, *x, *w;   // x [dim][n], w [n]
    const double *wsum;            // sum of w
    float *grad;                   // [n_params], zeroed
    double *loss;                  // zeroed
    int64_t n;
    int64_t max_layer;             // floats of the largest staged layer (the scratch follows)
    int dim, n_layers;
};

__global__ void nsf_wsum_kernel(const float *w, int64_t n, double *wsum) {
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        s += w[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(wsum, s);
}

// one layer's weights into shared memory in the staged layout (layer_at)
__device__ void stage_layer(const float *lp, int n_keep, int n_move, float *wsm) {
    const int64_t head = head_floats(n_keep);
    const int row = n_move * kParamsPerDim;
    __syncthreads();                                         // the previous layer's weights are consumed
    for (int64_t k = threadIdx.x; k < head; k += blockDim.x) wsm[k] = __ldg(lp + k);
    for (int64_t k = threadIdx.x; k < (int64_t)(kHidden + 1) * n_move * kPad; k += blockDim.x) {
        const int q = (int)(k % kPad);
        const int64_t rm = k / kPad;
        const int r = (int)(rm / n_move), m = (int)(rm % n_move);
        wsm[head + k] = q < kParamsPerDim ? __ldg(lp + head + (int64_t)r * row + m * kParamsPerDim + q) : 0.0f;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(128) nsf_grad_kernel(const NsfGradArgs a) {
    extern __shared__ __align__(16) float wsm[];
    // the warps' accumulation scratch after the layer's weights (max_layer floats)
    float *acc_scratch = wsm + a.max_layer + (threadIdx.x >> 5) * 2 * 32 * kAccRow;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = i < a.n;
    const int D = a.dim, half = D / 2;
    const float c = valid ? (float)(-(double)a.w[i] / *a.wsum) : 0.0f;     // d loss / d log q_i
    float v[kMaxDim];
#pragma unroll
    for (int j = 0; j < kMaxDim; ++j) v[j] = (valid && j < D) ? a.x[(int64_t)j * a.n + i] : 0.5f;
    float vin[kGradMaxLayers][kMaxDim];
    float logq = 0.0f;
    for (int layer = a.n_layers - 1; layer >= 0; --layer) {
        const int n_keep = layer % 2 == 0 ? half : D - half;
        stage_layer(a.params + layer_offset(layer, D), n_keep, D - n_keep, wsm);
#pragma unroll
        for (int j = 0; j < kMaxDim; ++j) vin[layer][j] = v[j];
        logq -= layer_inverse(layer_at(wsm, layer, D), v);
    }
    {
        float l = valid ? c * logq : 0.0f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
        if ((threadIdx.x & 31) == 0) atomicAdd(a.loss, (double)l);
    }
    float vbar[kMaxDim];
#pragma unroll
    for (int j = 0; j < kMaxDim; ++j) vbar[j] = 0.0f;       // z does not enter the loss
    for (int layer = 0; layer < a.n_layers; ++layer) {
        const int n_keep = layer % 2 == 0 ? half : D - half;
        const int64_t off = layer_offset(layer, D);
        stage_layer(a.params + off, n_keep, D - n_keep, wsm);
        float xin[kMaxDim];
#pragma unroll
        for (int j = 0; j < kMaxDim; ++j) xin[j] = vin[layer][j];
        WarpAtomicAcc acc{a.grad + off, acc_scratch};
        layer_backward(layer_at(wsm, layer, D), xin, vbar, c, acc);
    }
}

}  // namespace

struct fd_nsf {
    int dim = 0, n_layers = 0, device = 0;
    int64_t n_params = 0, max_layer = 0;
    float *d_params = nullptr;
    double *d_wsum = nullptr;      // the loss's weight normaliser (fd_nsf_kl_grad)
    // training state (fd_nsf_train): gradient, Adam moments, loss of each step
    float *d_grad = nullptr, *d_m = nullptr, *d_v = nullptr;
    double *d_loss = nullptr;
    int64_t step = 0;
    int tensor_path = 1;           // sampling / density: 1 conditioner on BF16 tensor cores, 0 FP32 CUDA cores
};

namespace {
fd_status nsf_sizes(int dim, int n_layers, int64_t &total, int64_t &max_layer) {
    total = 0;
    max_layer = 0;
    for (int l = 0; l < n_layers; ++l) {
        const int n_keep = l % 2 == 0 ? dim / 2 : dim - dim / 2;
        total += layer_floats(n_keep, dim - n_keep);
        max_layer = std::max(max_layer, layer_smem_floats(n_keep, dim - n_keep));
    }
    return FD_OK;
}

fd_status nsf_launch(const fd_nsf *f, bool inverse, const float *z, int64_t ldz, uint64_t seed, uint64_t iter,
                     int32_t inst, int64_t n, float *x, int64_t ldx, float *logq, cudaStream_t stream,
                     bool inv_q = false) {
    FD_REQUIRE(f && x && logq, "flow, x and logq are required");
    FD_REQUIRE(n > 0 && n <= (int64_t(1) << 36), "n must be in [1, 2^36]");
    FD_REQUIRE(inst >= 0 && inst < (1 << 24), "inst out of range");
    int dev = 0;
    FD_CHECK_CUDA(cudaGetDevice(&dev));
    FD_REQUIRE(dev == f->device, "flow belongs to another device");
    NsfArgs a;
    a.params = f->d_params;
    a.z = z;
    a.x = x;
    a.logq = logq;
    a.inv_q = inv_q ? 1 : 0;
    a.n = n;
    a.ldz = ldz;
    a.ldx = ldx;
    a.dim = f->dim;
    a.n_layers = f->n_layers;
    a.seed_lo = (uint32_t)seed;
    a.seed_hi = (uint32_t)(seed >> 32);
    a.iter = (uint32_t)iter;
    a.inst = (uint32_t)inst;
    if (f->tensor_path == 1) {
        const unsigned grid = (unsigned)((n + nsf_tc::BLOCK - 1) / nsf_tc::BLOCK);
        if (inverse) {
            FD_CHECK_CUDA(cudaFuncSetAttribute(nsf_tc_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)nsf_tc::SMEM));
            nsf_tc_kernel<true><<<grid, nsf_tc::THREADS, nsf_tc::SMEM, stream>>>(a);
        } else {
            FD_CHECK_CUDA(cudaFuncSetAttribute(nsf_tc_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)nsf_tc::SMEM));
            nsf_tc_kernel<false><<<grid, nsf_tc::THREADS, nsf_tc::SMEM, stream>>>(a);
        }
        FD_CHECK_CUDA(cudaGetLastError());
        return FD_OK;
    }
    const size_t smem = (size_t)f->max_layer * sizeof(float);
    if (inverse) {
        FD_CHECK_CUDA(cudaFuncSetAttribute(nsf_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        nsf_kernel<true><<<(unsigned)((n + 127) / 128), 128, smem, stream>>>(a);
    } else {
        FD_CHECK_CUDA(cudaFuncSetAttribute(nsf_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        nsf_kernel<false><<<(unsigned)((n + 127) / 128), 128, smem, stream>>>(a);
    }
    FD_CHECK_CUDA(cudaGetLastError());
    return FD_OK;
}
}  // namespace

extern "C" fd_status fd_nsf_create(int32_t dim, int32_t n_layers, fd_nsf **out) {
    FD_REQUIRE(out, "out is required");
    FD_REQUIRE(dim >= 2 && dim <= kMaxDim, "dim must be in [2, 24]");
    FD_REQUIRE(n_layers >= 1 && n_layers <= 64, "n_layers must be in [1, 64]");
    fd_nsf *f = new fd_nsf;
    f->dim = dim;
    f->n_layers = n_layers;
    nsf_sizes(dim, n_layers, f->n_params, f->max_layer);
    cudaError_t e = cudaGetDevice(&f->device);
    if (e == cudaSuccess) e = cudaMalloc(&f->d_params, (size_t)f->n_params * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(f->d_params, 0, (size_t)f->n_params * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&f->d_wsum, sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&f->d_grad, (size_t)f->n_params * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&f->d_m, (size_t)f->n_params * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&f->d_v, (size_t)f->n_params * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(f->d_m, 0, (size_t)f->n_params * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(f->d_v, 0, (size_t)f->n_params * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&f->d_loss, kNsfMaxTrainSteps * sizeof(double));
    if (e != cudaSuccess) {
        for (void *q : {(void *)f->d_params, (void *)f->d_wsum, (void *)f->d_grad, (void *)f->d_m, (void *)f->d_v,
                        (void *)f->d_loss})
            if (q) cudaFree(q);
        delete f;
        return fd::cuda_error(e, "creating a spline flow");
    }
    *out = f;
    return FD_OK;
}

extern "C" void fd_nsf_free(fd_nsf *f) {
    if (!f) return;
    for (void *q : {(void *)f->d_params, (void *)f->d_wsum, (void *)f->d_grad, (void *)f->d_m, (void *)f->d_v,
                    (void *)f->d_loss})
        if (q) cudaFree(q);
    delete f;
}

extern "C" int64_t fd_nsf_param_count(const fd_nsf *f) { return f ? f->n_params : 0; }

extern "C" fd_status fd_nsf_set_params(fd_nsf *f, const float *params, int64_t n) {
    FD_REQUIRE(f && params, "flow and params are required");
    FD_REQUIRE(n == f->n_params, "parameter count differs from fd_nsf_param_count");
    for (int64_t k = 0; k < n; ++k) FD_REQUIRE(std::isfinite(params[k]), "non-finite parameter");
    FD_CHECK_CUDA(cudaMemcpy(f->d_params, params, (size_t)n * sizeof(float), cudaMemcpyHostToDevice));
    FD_CHECK_CUDA(cudaMemset(f->d_m, 0, (size_t)n * sizeof(float)));     // a fresh Adam state
    FD_CHECK_CUDA(cudaMemset(f->d_v, 0, (size_t)n * sizeof(float)));
    f->step = 0;
    return FD_OK;
}

extern "C" fd_status fd_nsf_set_tensor_path(fd_nsf *f, int32_t path) {
    FD_REQUIRE(f, "null flow");
    FD_REQUIRE(path == 0 || path == 1, "path must be 0 (FP32 CUDA cores) or 1 (BF16 tensor cores)");
    f->tensor_path = path;
    return FD_OK;
}

extern "C" fd_status fd_nsf_forward(const fd_nsf *f, const float *z, int64_t n, float *x, float *logq,
                                    void *stream) {
    FD_REQUIRE(z, "z is required");
    return nsf_launch(f, false, z, n, 0, 0, 0, n, x, n, logq, (cudaStream_t)stream);
}

extern "C" fd_status fd_nsf_log_density(const fd_nsf *f, const float *x, int64_t n, float *z, float *logq,
                                        void *stream) {
    FD_REQUIRE(x && z, "x and z are required");
    return nsf_launch(f, true, x, n, 0, 0, 0, n, z, n, logq, (cudaStream_t)stream);
}

extern "C" fd_status fd_nsf_sample(const fd_nsf *f, uint64_t seed, uint64_t iter, int32_t inst, int64_t n, float *x,
                                   float *logq, void *stream) {
    return nsf_launch(f, false, nullptr, 0, seed, iter, inst, n, x, n, logq, (cudaStream_t)stream);
}

extern "C" fd_status fd_nsf_sample_w(const fd_nsf *f, uint64_t seed, uint64_t iter, int32_t inst, int64_t n, float *x,
                                     float *w, void *stream) {
    return nsf_launch(f, false, nullptr, 0, seed, iter, inst, n, x, n, w, (cudaStream_t)stream, true);
}

namespace {
fd_status kl_grad_impl(const fd_nsf *f, const float *x, const float *w, int64_t n, float *grad, double *loss,
                       cudaStream_t st) {
    FD_REQUIRE(f && x && w && grad && loss, "flow, x, w, grad and loss are required");
    FD_REQUIRE(n > 0 && n <= (int64_t(1) << 36), "n must be in [1, 2^36]");
    FD_REQUIRE(f->n_layers <= kGradMaxLayers, "the gradient pass supports at most 16 layers");
    int dev = 0;
    FD_CHECK_CUDA(cudaGetDevice(&dev));
    FD_REQUIRE(dev == f->device, "flow belongs to another device");
    FD_CHECK_CUDA(cudaMemsetAsync(grad, 0, (size_t)f->n_params * sizeof(float), st));
    FD_CHECK_CUDA(cudaMemsetAsync(loss, 0, sizeof(double), st));
    FD_CHECK_CUDA(cudaMemsetAsync(f->d_wsum, 0, sizeof(double), st));
    nsf_wsum_kernel<<<256, 256, 0, st>>>(w, n, f->d_wsum);
    FD_CHECK_CUDA(cudaGetLastError());
    NsfGradArgs a;
    a.params = f->d_params;
    a.x = x;
    a.w = w;
    a.wsum = f->d_wsum;
    a.grad = grad;
    a.loss = loss;
    a.n = n;
    a.max_layer = (f->max_layer + 3) / 4 * 4;
    a.dim = f->dim;
    a.n_layers = f->n_layers;
    const size_t smem = ((size_t)a.max_layer + 4 * 2 * 32 * kAccRow) * sizeof(float);
    FD_CHECK_CUDA(cudaFuncSetAttribute(nsf_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    nsf_grad_kernel<<<(unsigned)((n + 127) / 128), 128, smem, st>>>(a);
    FD_CHECK_CUDA(cudaGetLastError());
    return FD_OK;
}

// Adam (Kingma and Ba, 2015) with bias correction; b1t = b1^step, b2t = b2^step
__global__ void nsf_adam_kernel(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                                float *__restrict__ v, int64_t n, float lr, float b1, float b2, float b1t, float b2t,
                                float eps) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const float gk = g[k];
    const float mk = b1 * m[k] + (1.0f - b1) * gk, vk = b2 * v[k] + (1.0f - b2) * gk * gk;
    m[k] = mk;
    v[k] = vk;
    p[k] -= lr * (mk / (1.0f - b1t)) / (sqrtf(vk / (1.0f - b2t)) + eps);
}
}  // namespace

extern "C" fd_status fd_nsf_kl_grad(const fd_nsf *f, const float *x, const float *w, int64_t n, float *grad,
                                    double *loss, void *stream) {
    return kl_grad_impl(f, x, w, n, grad, loss, (cudaStream_t)stream);
}

extern "C" fd_status fd_nsf_train(fd_nsf *f, const float *x, const float *w, int64_t n, int32_t steps, float lr,
                                  double *loss_out, void *stream) {
    FD_REQUIRE(f && x && w, "flow, x and w are required");
    FD_REQUIRE(steps >= 1 && steps <= kNsfMaxTrainSteps, "steps must be in [1, 4096]");
    FD_REQUIRE(lr > 0.0f && std::isfinite(lr), "a positive learning rate is required");
    const cudaStream_t st = (cudaStream_t)stream;
    for (int k = 0; k < steps; ++k) {
        const fd_status s = kl_grad_impl(f, x, w, n, f->d_grad, f->d_loss + k, st);
        if (s != FD_OK) return s;
        f->step += 1;
        const float b1t = (float)std::pow(0.9, (double)f->step), b2t = (float)std::pow(0.999, (double)f->step);
        nsf_adam_kernel<<<(unsigned)((f->n_params + 255) / 256), 256, 0, st>>>(
            f->d_params, f->d_grad, f->d_m, f->d_v, f->n_params, lr, 0.9f, 0.999f, b1t, b2t, 1e-8f);
        FD_CHECK_CUDA(cudaGetLastError());
    }
    if (loss_out) {
        FD_CHECK_CUDA(cudaMemcpyAsync(loss_out, f->d_loss, steps * sizeof(double), cudaMemcpyDeviceToHost, st));
        FD_CHECK_CUDA(cudaStreamSynchronize(st));
    }
    return FD_OK;
}

extern "C" fd_status fd_nsf_get_params(const fd_nsf *f, float *params, int64_t n) {
    FD_REQUIRE(f && params && n == f->n_params, "params must hold fd_nsf_param_count floats");
    FD_CHECK_CUDA(cudaDeviceSynchronize());
    FD_CHECK_CUDA(cudaMemcpy(params, f->d_params, (size_t)n * sizeof(float), cudaMemcpyDeviceToHost));
    return FD_OK;
}
