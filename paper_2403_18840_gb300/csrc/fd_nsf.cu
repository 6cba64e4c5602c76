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
#include "fd_internal.cuh"

#include <algorithm>
#include <cmath>
#include <vector>

namespace {

constexpr int kBins = 8;
constexpr int kHidden = 32;
constexpr int kParamsPerDim = 3 * kBins - 1;
constexpr int kMaxDim = 24;
constexpr float kMinW = 1e-3f, kMinH = 1e-3f, kMinD = 1e-3f;
constexpr int kPad = 24;                 // a coordinate's 23 spline parameters, padded for 16-byte loads

// per layer: W0 [n_keep][32], b0 [32], two blocks of (Wa [32][32], ba [32],
// Wb [32][32], bb [32]), W1 [32][n_move * 23], b1 [n_move * 23]
__host__ __device__ __forceinline__ int64_t layer_floats(int n_keep, int n_move) {
    return (int64_t)n_keep * kHidden + kHidden + 2 * (2 * (kHidden * kHidden + kHidden)) +
           (int64_t)kHidden * n_move * kParamsPerDim + (int64_t)n_move * kParamsPerDim;
}

__device__ __forceinline__ float softplusf(float a) { return a > 20.0f ? a : log1pf(expf(a)); }

// The bin of the rational-quadratic spline on [0, 1] that holds v (an input
// coordinate, or with BY_Y an output coordinate) from the 23 parameters
// (widths, heights, internal-knot derivative logits): its knots and the
// derivatives there.
template <bool BY_Y>
__device__ __forceinline__ void rq_bin(const float (&p)[kPad], float v, float &x0, float &x1, float &y0, float &y1,
                                       float &d0, float &d1) {
    float mw = p[0], mh = p[kBins];
#pragma unroll
    for (int k = 1; k < kBins; ++k) {
        mw = fmaxf(mw, p[k]);
        mh = fmaxf(mh, p[kBins + k]);
    }
    float ew[kBins], eh[kBins], sw = 0.0f, sh = 0.0f;
#pragma unroll
    for (int k = 0; k < kBins; ++k) {
        ew[k] = expf(p[k] - mw);
        eh[k] = expf(p[kBins + k] - mh);
        sw += ew[k];
        sh += eh[k];
    }
    const float cw = (1.0f - kMinW * kBins) / sw, ch = (1.0f - kMinH * kBins) / sh;
    float xs[kBins + 1], ys[kBins + 1];
    xs[0] = 0.0f;
    ys[0] = 0.0f;
#pragma unroll
    for (int k = 0; k < kBins; ++k) {
        xs[k + 1] = xs[k] + (kMinW + cw * ew[k]);
        ys[k + 1] = ys[k] + (kMinH + ch * eh[k]);
    }
    xs[kBins] = 1.0f;
    ys[kBins] = 1.0f;
    int bin = 0;                                   // the number of internal knots at or below v
#pragma unroll
    for (int k = 1; k < kBins; ++k) bin += v >= (BY_Y ? ys[k] : xs[k]) ? 1 : 0;
    x0 = 0.0f;
    x1 = 1.0f;
    y0 = 0.0f;
    y1 = 1.0f;
#pragma unroll
    for (int k = 0; k < kBins; ++k)
        if (k == bin) {
            x0 = xs[k];
            x1 = xs[k + 1];
            y0 = ys[k];
            y1 = ys[k + 1];
        }
    float pd0 = 0.0f, pd1 = 0.0f;                // the derivative logits at the bin's knots
#pragma unroll
    for (int k = 0; k < kBins - 1; ++k) {
        if (k == bin - 1) pd0 = p[2 * kBins + k];
        if (k == bin) pd1 = p[2 * kBins + k];
    }
    d0 = bin > 0 ? kMinD + softplusf(pd0) : 1.0f;
    d1 = bin < kBins - 1 ? kMinD + softplusf(pd1) : 1.0f;
}

// log g' at the bin's relative position xi
__device__ __forceinline__ float rq_logd(float s, float xi, float d0, float d1) {
    const float t = xi * (1.0f - xi), den = s + (d1 + d0 - 2.0f * s) * t;
    const float num = s * s * (d1 * xi * xi + 2.0f * s * t + d0 * (1.0f - xi) * (1.0f - xi));
    return logf(num) - 2.0f * logf(den);
}

// y = g(u) and log g'(u)
__device__ __forceinline__ void rq_spline(const float (&p)[kPad], float u, float &y, float &logd) {
    float x0, x1, y0, y1, d0, d1;
    rq_bin<false>(p, u, x0, x1, y0, y1, d0, d1);
    const float wk = x1 - x0, hk = y1 - y0;
    const float s = hk / wk, xi = (u - x0) / wk, t = xi * (1.0f - xi);
    const float den = s + (d1 + d0 - 2.0f * s) * t;
    y = y0 + hk * (s * xi * xi + d0 * t) / den;
    logd = rq_logd(s, xi, d0, d1);
}

// u = g^-1(y) (the root in [0, 1] of the bin's quadratic in xi) and log g'(u)
__device__ __forceinline__ void rq_spline_inverse(const float (&p)[kPad], float y, float &u, float &logd) {
    float x0, x1, y0, y1, d0, d1;
    rq_bin<true>(p, y, x0, x1, y0, y1, d0, d1);
    const float wk = x1 - x0, hk = y1 - y0, s = hk / wk, dy = y - y0, e = d1 + d0 - 2.0f * s;
    const float qa = hk * (s - d0) + dy * e, qb = hk * d0 - dy * e, qc = -s * dy;
    const float disc = fmaxf(qb * qb - 4.0f * qa * qc, 0.0f);
    const float xi = (2.0f * qc) / (-qb - sqrtf(disc));
    u = x0 + xi * wk;
    logd = rq_logd(s, xi, d0, d1);
}

struct NsfArgs {
    const float *params;      // all layers, in order
    const float *z;           // [dim][ldz] or null: Philox stream
    float *x;                 // [dim][ldx]
    float *logq;              // [n]
    int64_t n, ldz, ldx;
    int dim, n_layers;
    uint32_t seed_lo, seed_hi, iter, inst;
};

// shared-memory layout of a layer: as in global memory up to the residual
// blocks; W1 and b1 re-laid as rows of kPad (23 parameters and a zero), so
// every weight row starts on 16 bytes and is read as float4

__host__ __device__ __forceinline__ int64_t head_floats(int n_keep) {
    return (int64_t)n_keep * kHidden + kHidden + 2 * (2 * (kHidden * kHidden + kHidden));
}

__host__ __device__ __forceinline__ int64_t layer_smem_floats(int n_keep, int n_move) {
    return head_floats(n_keep) + (int64_t)(kHidden + 1) * n_move * kPad;
}

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
        const float *lp = a.params;
        for (int l = 0; l < layer; ++l) lp += layer_floats(l % 2 == 0 ? half : D - half, l % 2 == 0 ? D - half : half);
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
    a.logq[i] = logq;
}

}  // namespace

struct fd_nsf {
    int dim = 0, n_layers = 0, device = 0;
    int64_t n_params = 0, max_layer = 0;
    float *d_params = nullptr;
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
                     int32_t inst, int64_t n, float *x, int64_t ldx, float *logq, cudaStream_t stream) {
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
    a.n = n;
    a.ldz = ldz;
    a.ldx = ldx;
    a.dim = f->dim;
    a.n_layers = f->n_layers;
    a.seed_lo = (uint32_t)seed;
    a.seed_hi = (uint32_t)(seed >> 32);
    a.iter = (uint32_t)iter;
    a.inst = (uint32_t)inst;
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
    if (e != cudaSuccess) {
        if (f->d_params) cudaFree(f->d_params);
        delete f;
        return fd::cuda_error(e, "creating a spline flow");
    }
    *out = f;
    return FD_OK;
}

extern "C" void fd_nsf_free(fd_nsf *f) {
    if (!f) return;
    if (f->d_params) cudaFree(f->d_params);
    delete f;
}

extern "C" int64_t fd_nsf_param_count(const fd_nsf *f) { return f ? f->n_params : 0; }

extern "C" fd_status fd_nsf_set_params(fd_nsf *f, const float *params, int64_t n) {
    FD_REQUIRE(f && params, "flow and params are required");
    FD_REQUIRE(n == f->n_params, "parameter count differs from fd_nsf_param_count");
    for (int64_t k = 0; k < n; ++k) FD_REQUIRE(std::isfinite(params[k]), "non-finite parameter");
    FD_CHECK_CUDA(cudaMemcpy(f->d_params, params, (size_t)n * sizeof(float), cudaMemcpyHostToDevice));
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
