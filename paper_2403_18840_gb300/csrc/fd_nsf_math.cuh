// Rational-quadratic spline coupling layers of the spline flow (App. A;
// Durkan et al., 2019): the spline, its inverse, its closed-form partial
// derivatives, and one coupling layer's conditioner, inverse and reverse-mode
// backward on one sample.  Plain FP32 functions callable on the device and on
// the host; the kernels in fd_nsf.cu stage a layer's weights in shared memory
// and call them per sample.
#pragma once

#include <math.h>
#include <stdint.h>

namespace nsf {

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

__host__ __device__ __forceinline__ float softplusf(float a) { return a > 20.0f ? a : log1pf(expf(a)); }

// The bin of the rational-quadratic spline on [0, 1] that holds v (an input
// coordinate, or with BY_Y an output coordinate) from the 23 parameters
// (widths, heights, internal-knot derivative logits): its knots and the
// derivatives there.
template <bool BY_Y>
__host__ __device__ __forceinline__ void rq_bin(const float (&p)[kPad], float v, float &x0, float &x1, float &y0, float &y1,
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
__host__ __device__ __forceinline__ float rq_logd(float s, float xi, float d0, float d1) {
    const float t = xi * (1.0f - xi), den = s + (d1 + d0 - 2.0f * s) * t;
    const float num = s * s * (d1 * xi * xi + 2.0f * s * t + d0 * (1.0f - xi) * (1.0f - xi));
    return logf(num) - 2.0f * logf(den);
}

// y = g(u) and log g'(u)
__host__ __device__ __forceinline__ void rq_spline(const float (&p)[kPad], float u, float &y, float &logd) {
    float x0, x1, y0, y1, d0, d1;
    rq_bin<false>(p, u, x0, x1, y0, y1, d0, d1);
    const float wk = x1 - x0, hk = y1 - y0;
    const float s = hk / wk, xi = (u - x0) / wk, t = xi * (1.0f - xi);
    const float den = s + (d1 + d0 - 2.0f * s) * t;
    y = y0 + hk * (s * xi * xi + d0 * t) / den;
    logd = rq_logd(s, xi, d0, d1);
}

// u = g^-1(y) (the root in [0, 1] of the bin's quadratic in xi) and log g'(u)
__host__ __device__ __forceinline__ void rq_spline_inverse(const float (&p)[kPad], float y, float &u, float &logd) {
    float x0, x1, y0, y1, d0, d1;
    rq_bin<true>(p, y, x0, x1, y0, y1, d0, d1);
    const float wk = x1 - x0, hk = y1 - y0, s = hk / wk, dy = y - y0, e = d1 + d0 - 2.0f * s;
    const float qa = hk * (s - d0) + dy * e, qb = hk * d0 - dy * e, qc = -s * dy;
    const float disc = fmaxf(qb * qb - 4.0f * qa * qc, 0.0f);
    const float xi = (2.0f * qc) / (-qb - sqrtf(disc));
    u = x0 + xi * wk;
    logd = rq_logd(s, xi, d0, d1);
}

// shared-memory layout of a layer: as in global memory up to the residual
// blocks; W1 and b1 re-laid as rows of kPad (23 parameters and a zero), so
// every weight row starts on 16 bytes and is read as float4

__host__ __device__ __forceinline__ int64_t head_floats(int n_keep) {
    return (int64_t)n_keep * kHidden + kHidden + 2 * (2 * (kHidden * kHidden + kHidden));
}

__host__ __device__ __forceinline__ int64_t layer_smem_floats(int n_keep, int n_move) {
    return head_floats(n_keep) + (int64_t)(kHidden + 1) * n_move * kPad;
}


// Closed-form partials of the spline at input u (in its bin, with knots from
// softmax widths/heights and softplus derivatives): gp = dg/dp and lp = dl/dp
// over the 23 parameters (index 23 is padding, 0), l_u = dl/du and l = log g'(u).
// g = y_k + h N/E and l = 2 log s + log M - 2 log E with s = h/w, xi = (u -
// x_k)/w, N = s xi^2 + d0 xi(1-xi), E = s + (d0 + d1 - 2s) xi(1-xi), M = d1
// xi^2 + 2 s xi(1-xi) + d0 (1-xi)^2; the chain rule through (x_k, w, y_k, h,
// d0, d1) to the parameters.
__host__ __device__ __forceinline__ void rq_partials(const float (&p)[kPad], float u, float (&gp)[kPad],
                                                     float (&lp)[kPad], float &l_u, float &l) {
    float mw = p[0], mh = p[kBins];
#pragma unroll
    for (int k = 1; k < kBins; ++k) {
        mw = fmaxf(mw, p[k]);
        mh = fmaxf(mh, p[kBins + k]);
    }
    float sw[kBins], sh[kBins], zw = 0.0f, zh = 0.0f;
#pragma unroll
    for (int k = 0; k < kBins; ++k) {
        sw[k] = expf(p[k] - mw);
        sh[k] = expf(p[kBins + k] - mh);
        zw += sw[k];
        zh += sh[k];
    }
#pragma unroll
    for (int k = 0; k < kBins; ++k) {
        sw[k] /= zw;                                   // softmax of the width and height logits
        sh[k] /= zh;
    }
    const float cw = 1.0f - kMinW * kBins, ch = 1.0f - kMinH * kBins;
    int bin = 0;
    float xs = 0.0f;
#pragma unroll
    for (int k = 1; k < kBins; ++k) {
        xs += kMinW + cw * sw[k - 1];
        bin += u >= xs ? 1 : 0;
    }
    float xk = 0.0f, w = 1.0f, h = 1.0f, swk = 0.0f, shk = 0.0f, below_w = 0.0f, below_h = 0.0f;
    float ys = 0.0f;
    xs = 0.0f;
#pragma unroll
    for (int k = 0; k < kBins; ++k) {
        const float wi = kMinW + cw * sw[k], hi = kMinH + ch * sh[k];
        if (k == bin) {
            xk = xs;
            w = k == kBins - 1 ? 1.0f - xs : wi;       // the last knot is exactly 1
            h = k == kBins - 1 ? 1.0f - ys : hi;
            swk = sw[k];
            shk = sh[k];
        }
        if (k < bin) {
            below_w += sw[k];
            below_h += sh[k];
        }
        xs += wi;
        ys += hi;
    }
    float pd0 = 0.0f, pd1 = 0.0f;
#pragma unroll
    for (int k = 0; k < kBins - 1; ++k) {
        if (k == bin - 1) pd0 = p[2 * kBins + k];
        if (k == bin) pd1 = p[2 * kBins + k];
    }
    const float d0 = bin > 0 ? kMinD + softplusf(pd0) : 1.0f, d1 = bin < kBins - 1 ? kMinD + softplusf(pd1) : 1.0f;
    const float sig0 = 1.0f / (1.0f + expf(-pd0)), sig1 = 1.0f / (1.0f + expf(-pd1));   // softplus'
    const float s = h / w, xi = (u - xk) / w, t = xi * (1.0f - xi), tp = 1.0f - 2.0f * xi, om = 1.0f - xi;
    const float N = s * xi * xi + d0 * t, E = s + (d1 + d0 - 2.0f * s) * t;
    const float M = d1 * xi * xi + 2.0f * s * t + d0 * om * om;
    l = 2.0f * logf(s) + logf(M) - 2.0f * logf(E);
    const float E2 = E * E;
    const float E_xi = (d1 + d0 - 2.0f * s) * tp, E_s = 1.0f - 2.0f * t;
    const float g_xi = h * ((2.0f * s * xi + d0 * tp) * E - N * E_xi) / E2;
    const float g_s = h * (xi * xi * E - N * E_s) / E2;
    const float g_d0 = h * (t * E - N * t) / E2, g_d1 = -h * N * t / E2;
    const float l_xi = (2.0f * d1 * xi + 2.0f * s * tp - 2.0f * d0 * om) / M - 2.0f * E_xi / E;
    const float l_s = 2.0f / s + 2.0f * t / M - 2.0f * E_s / E;
    const float l_d0 = om * om / M - 2.0f * t / E, l_d1 = xi * xi / M - 2.0f * t / E;
    // through x_k (xi), w (xi and s), h (s and the factor h), y_k
    const float g_xk = -g_xi / w, l_xk = -l_xi / w;
    const float g_w = -(g_xi * xi + g_s * s) / w, l_w = -(l_xi * xi + l_s * s) / w;
    const float g_h = N / E + g_s / w, l_h = l_s / w;
    l_u = l_xi / w;
#pragma unroll
    for (int a = 0; a < kBins; ++a) {
        // d(softmax_j)/d(logit_a) = sm_j (delta_ja - sm_a)
        const float dxk = cw * ((a < bin ? sw[a] : 0.0f) - below_w * sw[a]);
        const float dw = cw * ((a == bin ? sw[a] : 0.0f) - swk * sw[a]);
        const float dyk = ch * ((a < bin ? sh[a] : 0.0f) - below_h * sh[a]);
        const float dh = ch * ((a == bin ? sh[a] : 0.0f) - shk * sh[a]);
        gp[a] = g_xk * dxk + g_w * dw;
        lp[a] = l_xk * dxk + l_w * dw;
        gp[kBins + a] = dyk + g_h * dh;
        lp[kBins + a] = l_h * dh;
    }
#pragma unroll
    for (int j = 0; j < kBins - 1; ++j) {
        gp[2 * kBins + j] = (j == bin - 1 ? g_d0 * sig0 : 0.0f) + (j == bin ? g_d1 * sig1 : 0.0f);
        lp[2 * kBins + j] = (j == bin - 1 ? l_d0 * sig0 : 0.0f) + (j == bin ? l_d1 * sig1 : 0.0f);
    }
    gp[kPad - 1] = 0.0f;
    lp[kPad - 1] = 0.0f;
}

// element j of a register-resident coordinate vector (runtime j, unrolled select)
__host__ __device__ __forceinline__ float sel(const float (&v)[kMaxDim], int j) {
    float r = 0.0f;
#pragma unroll
    for (int q = 0; q < kMaxDim; ++q)
        if (q == j) r = v[q];
    return r;
}

__host__ __device__ __forceinline__ void put(float (&v)[kMaxDim], int j, float x) {
#pragma unroll
    for (int q = 0; q < kMaxDim; ++q)
        if (q == j) v[q] = x;
}

// One coupling layer's weights in the staged layout (head as in the
// parameter vector, W1/b1 as rows of kPad) and which coordinates it keeps.
struct Layer {
    const float *W0, *b0, *blk, *W1, *b1;
    int n_keep, n_move, keep0, move0;
};

__host__ __device__ __forceinline__ Layer layer_at(const float *staged, int layer, int dim) {
    const int half = dim / 2;
    Layer L;
    L.n_keep = layer % 2 == 0 ? half : dim - half;
    L.n_move = dim - L.n_keep;
    L.keep0 = layer % 2 == 0 ? 0 : half;
    L.move0 = layer % 2 == 0 ? half : 0;
    L.W0 = staged;
    L.b0 = L.W0 + L.n_keep * kHidden;
    L.blk = L.b0 + kHidden;
    L.W1 = staged + head_floats(L.n_keep);
    L.b1 = L.W1 + (int64_t)kHidden * L.n_move * kPad;
    return L;
}

// the parameter vector's offset of layer `layer` (layers alternate n_keep)
__host__ __device__ __forceinline__ int64_t layer_offset(int layer, int dim) {
    const int half = dim / 2;
    int64_t o = 0;
    for (int l = 0; l < layer; ++l) o += layer_floats(l % 2 == 0 ? half : dim - half, l % 2 == 0 ? dim - half : half);
    return o;
}

// The conditioner on the kept coordinates of x: h0 = W0 x + b0, then two
// residual blocks h <- h + Wb relu(Wa relu(h) + ba) + bb; t0, t1 are the
// blocks' inner pre-activations and h2 the output features.
__host__ __device__ __forceinline__ void conditioner(const Layer &L, const float (&x)[kMaxDim], float (&h0)[kHidden],
                                                     float (&t0)[kHidden], float (&h1)[kHidden],
                                                     float (&t1)[kHidden], float (&h2)[kHidden]) {
    for (int q = 0; q < kHidden; ++q) h0[q] = L.b0[q];
    for (int r = 0; r < L.n_keep; ++r) {
        const float xv = sel(x, L.keep0 + r);
        for (int q = 0; q < kHidden; ++q) h0[q] = fmaf(xv, L.W0[r * kHidden + q], h0[q]);
    }
    for (int bk = 0; bk < 2; ++bk) {
        const float *Wa = L.blk + bk * 2 * (kHidden * kHidden + kHidden), *ba = Wa + kHidden * kHidden;
        const float *Wb = ba + kHidden, *bb = Wb + kHidden * kHidden;
        const float(&hin)[kHidden] = bk == 0 ? h0 : h1;
        float(&tt)[kHidden] = bk == 0 ? t0 : t1;
        float(&hout)[kHidden] = bk == 0 ? h1 : h2;
        for (int q = 0; q < kHidden; ++q) tt[q] = ba[q];
        for (int r = 0; r < kHidden; ++r) {
            const float a = fmaxf(hin[r], 0.0f);
            for (int q = 0; q < kHidden; ++q) tt[q] = fmaf(a, Wa[r * kHidden + q], tt[q]);
        }
        for (int q = 0; q < kHidden; ++q) hout[q] = bb[q];
        for (int r = 0; r < kHidden; ++r) {
            const float b = fmaxf(tt[r], 0.0f);
            for (int q = 0; q < kHidden; ++q) hout[q] = fmaf(b, Wb[r * kHidden + q], hout[q]);
        }
        for (int q = 0; q < kHidden; ++q) hout[q] += hin[q];
    }
}

// the 23 spline parameters of moved coordinate m: b1 + W1^T h2
__host__ __device__ __forceinline__ void spline_params(const Layer &L, const float (&h2)[kHidden], int m,
                                                       float (&p)[kPad]) {
    for (int q = 0; q < kPad; ++q) p[q] = L.b1[m * kPad + q];
    for (int r = 0; r < kHidden; ++r)
        for (int q = 0; q < kPad; ++q) p[q] = fmaf(h2[r], L.W1[(r * L.n_move + m) * kPad + q], p[q]);
}

// The layer's inverse on v in place; returns the sum of the moved
// coordinates' log g'(u).
__host__ __device__ __forceinline__ float layer_inverse(const Layer &L, float (&v)[kMaxDim]) {
    float h0[kHidden], t0[kHidden], h1[kHidden], t1[kHidden], h2[kHidden];
    conditioner(L, v, h0, t0, h1, t1, h2);
    float sum = 0.0f;
    for (int m = 0; m < L.n_move; ++m) {
        float p[kPad], u, ld;
        spline_params(L, h2, m, p);
        rq_spline_inverse(p, fminf(fmaxf(sel(v, L.move0 + m), 0.0f), 1.0f), u, ld);
        put(v, L.move0 + m, u);
        sum += ld;
    }
    return sum;
}

// Gradient accumulation of layer_backward: the rank-one updates
// G[r][q] += a[r] b[q] (r < na, q < nb) at offset off + r stride + q and the
// vector updates G[q] += b[q] at off + q, by default through the accumulator's
// scalar call acc(k, value); an accumulator type may overload these two (the
// device one sums a warp's 32 samples through shared memory).
template <class Acc, int NA, int NB>
__host__ __device__ __forceinline__ void acc_outer(Acc &acc, int64_t off, int64_t stride, const float (&a)[NA],
                                                   int na, const float (&b)[NB], int nb) {
    for (int r = 0; r < na; ++r)
        for (int q = 0; q < nb; ++q) acc(off + r * stride + q, a[r] * b[q]);
}
template <class Acc, int NB>
__host__ __device__ __forceinline__ void acc_vec(Acc &acc, int64_t off, const float (&b)[NB], int nb) {
    for (int q = 0; q < nb; ++q) acc(off + q, b[q]);
}

// Reverse mode through one layer's inverse on one sample.  xin is the
// layer's input (the point on the x side), vbar on entry the loss's adjoint
// of the layer's output and on exit that of its input; c = d loss / d log q
// (the sample's -w / sum w, 0 for a padding thread).  Every parameter
// gradient goes to the accumulator (acc_outer / acc_vec above), offsets
// within the layer's slice of the parameter vector.  On the device all lanes
// of a warp make the same sequence of accumulator calls.
#pragma nv_exec_check_disable
template <class Acc>
__host__ __device__ __forceinline__ void layer_backward(const Layer &L, const float (&xin)[kMaxDim],
                                                        float (&vbar)[kMaxDim], float c, Acc &acc) {
    float h0[kHidden], t0[kHidden], h1[kHidden], t1[kHidden], h2[kHidden], hbar[kHidden];
    conditioner(L, xin, h0, t0, h1, t1, h2);
    const int64_t oW1 = head_floats(L.n_keep), ob1 = oW1 + (int64_t)kHidden * L.n_move * kParamsPerDim;
    for (int q = 0; q < kHidden; ++q) hbar[q] = 0.0f;
    // the splines: loss = ... - c l(u, p), u = g^-1(y; p), du/dy = 1/g', du/dp = -(dg/dp)/g'
    for (int m = 0; m < L.n_move; ++m) {
        float p[kPad], u, ld, gp[kPad], lpp[kPad], l_u, l;
        spline_params(L, h2, m, p);
        rq_spline_inverse(p, fminf(fmaxf(sel(xin, L.move0 + m), 0.0f), 1.0f), u, ld);
        rq_partials(p, u, gp, lpp, l_u, l);
        const float inv_g = expf(-l);
        const float ubar = c == 0.0f ? 0.0f : sel(vbar, L.move0 + m) - c * l_u;
        float pbar[kPad];
        for (int q = 0; q < kPad; ++q) pbar[q] = c == 0.0f ? 0.0f : -c * lpp[q] - ubar * inv_g * gp[q];
        put(vbar, L.move0 + m, ubar * inv_g);
        acc_vec(acc, ob1 + m * kParamsPerDim, pbar, kParamsPerDim);
        acc_outer(acc, oW1 + m * kParamsPerDim, (int64_t)L.n_move * kParamsPerDim, h2, kHidden, pbar,
                  kParamsPerDim);
        for (int r = 0; r < kHidden; ++r) {
            float s = 0.0f;
            for (int q = 0; q < kParamsPerDim; ++q) s = fmaf(pbar[q], L.W1[(r * L.n_move + m) * kPad + q], s);
            hbar[r] += s;
        }
    }
    // the residual blocks, last first
    for (int bk = 1; bk >= 0; --bk) {
        const int64_t oWa = (int64_t)L.n_keep * kHidden + kHidden + bk * 2 * (kHidden * kHidden + kHidden);
        const int64_t oba = oWa + kHidden * kHidden, oWb = oba + kHidden, obb = oWb + kHidden * kHidden;
        const float *Wa = L.W0 + oWa, *Wb = L.W0 + oWb;
        const float(&hin)[kHidden] = bk == 0 ? h0 : h1;
        const float(&tt)[kHidden] = bk == 0 ? t0 : t1;
        float tbar[kHidden], hadd[kHidden], relu_t[kHidden], relu_h[kHidden];
        for (int q = 0; q < kHidden; ++q) {
            relu_t[q] = fmaxf(tt[q], 0.0f);
            relu_h[q] = fmaxf(hin[q], 0.0f);
        }
        acc_vec(acc, obb, hbar, kHidden);
        acc_outer(acc, oWb, kHidden, relu_t, kHidden, hbar, kHidden);
        for (int r = 0; r < kHidden; ++r) {
            float s = 0.0f;
            for (int q = 0; q < kHidden; ++q) s = fmaf(hbar[q], Wb[r * kHidden + q], s);
            tbar[r] = tt[r] > 0.0f ? s : 0.0f;
        }
        acc_vec(acc, oba, tbar, kHidden);
        acc_outer(acc, oWa, kHidden, relu_h, kHidden, tbar, kHidden);
        for (int r = 0; r < kHidden; ++r) {
            float s = 0.0f;
            for (int q = 0; q < kHidden; ++q) s = fmaf(tbar[q], Wa[r * kHidden + q], s);
            hadd[r] = hin[r] > 0.0f ? s : 0.0f;
        }
        for (int q = 0; q < kHidden; ++q) hbar[q] += hadd[q];
    }
    // the input map: kept coordinates pass through and feed h0
    const int64_t ob0 = (int64_t)L.n_keep * kHidden;
    float xk[kMaxDim / 2];
    for (int r = 0; r < kMaxDim / 2; ++r) xk[r] = r < L.n_keep ? sel(xin, L.keep0 + r) : 0.0f;
    acc_vec(acc, ob0, hbar, kHidden);
    acc_outer(acc, 0, kHidden, xk, L.n_keep, hbar, kHidden);
    for (int r = 0; r < L.n_keep; ++r) {
        float s = 0.0f;
        for (int q = 0; q < kHidden; ++q) s = fmaf(hbar[q], L.W0[r * kHidden + q], s);
        put(vbar, L.keep0 + r, sel(vbar, L.keep0 + r) + s);
    }
}

}  // namespace nsf
