// Device runtime shared by the tape interpreter and the specialised
// (straight-line) integrand kernels.  The specialised kernels are compiled at
// run time by NVRTC, which sees this file as an in-memory header, so it
// includes nothing and uses only the CUDA built-ins.
//
// What one sample computes (Eq. sigma_integration with the counterterm
// expansion of Eq. sigma_xi_dmu_dlambda): Philox uniforms -> sampler map ->
// loop momenta and interaction times (Sec. IV, spherical coordinates with a
// momentum cutoff) -> leaf Taylor families of G0 and V (Eq. taylor_node) ->
// contraction -> every root weighted by its Jacobian and exp(i pi x_out).
#pragma once

#ifdef __CUDACC_RTC__
typedef unsigned char uint8_t;
typedef int int32_t;
typedef unsigned int uint32_t;
typedef long long int64_t;
typedef unsigned long long uint64_t;
#else
#include <stdint.h>
#endif

constexpr int FD_MAX_ORDER = 6;
constexpr int FD_MAX_DIM = 4 * FD_MAX_ORDER - 1;
constexpr int FD_MAX_M = 7;         // largest Taylor order of a leaf family (incl. d/dk)
constexpr int FD_MAX_INST = 256;    // instances per launch (kernel-parameter descriptors)
constexpr float FD_INV_2PI2 = 0.050660591821168885f;   // 1 / (2 pi^2)
constexpr float FD_8PI = 25.132741228718345f;

// ---- launch descriptors (identical layout in every compilation) -------------
struct InstDesc {
    const uint64_t *tape;      // instruction words (device; interpreter only)
    const uint32_t *roots;     // root table (device): n | m<<8 | l<<16 | dk<<24, 0
    const float *edges;        // VEGAS FP32 edges [dim][nb+1] or null
    double *hist;              // VEGAS histogram [dim][nb] or null
    const float *points;       // explicit points [dim_max][n] or null
    const float *point_w;      // explicit weights [n] or null
    int32_t n_instr, n_slots, order, dim, n_roots, n_bins;
    float kext, mu, beta, Lambda, kc;
    int32_t id;                // instance index of the call (partials, per-sample rows, Philox stream)
};

struct EvalArgs {
    int32_t n_inst, tiles_per_inst, r_max, slots_total, dim_max;
    int32_t hist_smem;                 // floats of dynamic shared memory for the tile histogram (0: none)
    int64_t n_per_inst, tile;
    uint32_t seed_lo, seed_hi, iter;
    const uint32_t *iter_dev;          // optional: iteration += *iter_dev (read on the device)
    unsigned long long *queue;         // work counter (reset to 0 before the launch)
    double *partials;
    float *per_sample_f;
    int *status;
    uint8_t perm[FD_MAX_INST];         // descriptors in decreasing cost: work items go heaviest first
    InstDesc inst[FD_MAX_INST];
};

// ---- Philox4x32-10 (Salmon et al., SC'11) ----------------------------------------
struct u32x4 {
    uint32_t x, y, z, w;
};

__device__ __forceinline__ u32x4 philox4x32_10(u32x4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x;
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = u32x4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// u = ((w >> 9) + 0.5) * 2^-23, exact in FP32, strictly inside (0, 1)
__device__ __forceinline__ float word_to_uniform(uint32_t w) {
    return __uint2float_rn(w >> 9) * 1.1920928955078125e-07f + 5.9604644775390625e-08f;
}

// Neumaier compensated addition: (s, c) += v
__device__ __forceinline__ void neumaier(double &s, double &c, double v) {
    const double t = s + v;
    if (fabs(s) >= fabs(v))
        c += (s - t) + v;
    else
        c += (v - t) + s;
    s = t;
}

// one MUFU reciprocal (relative error about 1 ulp); the arguments here are
// normal numbers well inside the FP32 range
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Two samples' values in one register pair: every arithmetic operation is one
// packed two-lane instruction (add, multiply, fused multiply-add; each lane
// rounds exactly as the scalar operation), so the code of a compilation unit is
// fetched and issued once for two samples.  Subtraction is a + (-1) b and
// negation (-1) a, both exact.  Scalars convert implicitly (both lanes).
struct FdF2 {
    float2 v;
    __device__ __forceinline__ FdF2() {}
    __device__ __forceinline__ FdF2(float s) : v(make_float2(s, s)) {}
    __device__ __forceinline__ FdF2(float a, float b) : v(make_float2(a, b)) {}
};
struct FdM2 {
    bool x, y;
};
__device__ __forceinline__ FdF2 fd_wrap(float2 v) {
    FdF2 r;
    r.v = v;
    return r;
}
__device__ __forceinline__ FdF2 operator+(FdF2 a, FdF2 b) { return fd_wrap(__fadd2_rn(a.v, b.v)); }
__device__ __forceinline__ FdF2 operator*(FdF2 a, FdF2 b) { return fd_wrap(__fmul2_rn(a.v, b.v)); }
__device__ __forceinline__ FdF2 operator-(FdF2 a, FdF2 b) {
    return fd_wrap(__ffma2_rn(b.v, make_float2(-1.0f, -1.0f), a.v));
}
__device__ __forceinline__ FdF2 operator-(FdF2 a) { return fd_wrap(__fmul2_rn(a.v, make_float2(-1.0f, -1.0f))); }
__device__ __forceinline__ float fd_fma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ FdF2 fd_fma(FdF2 a, FdF2 b, FdF2 c) { return fd_wrap(__ffma2_rn(a.v, b.v, c.v)); }
__device__ __forceinline__ float fd_abs(float a) { return fabsf(a); }
__device__ __forceinline__ FdF2 fd_abs(FdF2 a) { return FdF2(fabsf(a.v.x), fabsf(a.v.y)); }
__device__ __forceinline__ float fd_exp(float a) { return __expf(a); }
__device__ __forceinline__ FdF2 fd_exp(FdF2 a) { return FdF2(__expf(a.v.x), __expf(a.v.y)); }
__device__ __forceinline__ bool fd_gt0(float a) { return a > 0.0f; }
__device__ __forceinline__ FdM2 fd_gt0(FdF2 a) { return FdM2{a.v.x > 0.0f, a.v.y > 0.0f}; }
__device__ __forceinline__ bool fd_lt0(float a) { return a < 0.0f; }
__device__ __forceinline__ FdM2 fd_lt0(FdF2 a) { return FdM2{a.v.x < 0.0f, a.v.y < 0.0f}; }
__device__ __forceinline__ float fd_sel(bool c, float a, float b) { return c ? a : b; }
__device__ __forceinline__ FdF2 fd_sel(FdM2 c, FdF2 a, FdF2 b) {
    return FdF2(c.x ? a.v.x : b.v.x, c.y ? a.v.y : b.v.y);
}
__device__ __forceinline__ FdF2 rcp_approx(FdF2 x) { return FdF2(rcp_approx(x.v.x), rcp_approx(x.v.y)); }

// 1 / (k + 1) for the Taylor recurrences (no division in the inner loops)
__device__ __forceinline__ float inv_int(int k1) {
    return k1 == 1 ? 1.0f : k1 == 2 ? 0.5f : k1 == 3 ? 0.33333334f : k1 == 4 ? 0.25f
         : k1 == 5 ? 0.2f : k1 == 6 ? 0.16666667f : k1 == 7 ? 0.14285715f : 0.125f;
}

// ---- leaf families (Eq. taylor_node) -------------------------------------------
// G0 Taylor family at momentum p (|p|^2 = p2, p_z = pz; ks = coefficient of
// k_ext in p) and hypercube time difference dx of its two interaction lines:
// c_j = (d/dmu)^j G0 / j!, j <= M, then (when dk) d c_j / d k_ext, j <= M.
// Written as sign * exp(-eps tau*) * phi(eps - dmu) with the Fermi factor
// phi >= 1/2 (phi = 1 - f for eps >= 0, f for eps < 0) and tau* the matching
// antiperiodic time, so the exponent is never positive.  The series of
// phi(eps - d) follows from the logistic ODE d phi / d eps = +-beta phi (1 - phi)
// (a Taylor-mode recurrence); the series of exp(d tau*) is tau*^k / k!.
// out(j, value) receives the (M + 1) (1 + dk) values.
template <class T, class Out>
__device__ __forceinline__ void g_family(T p2, T pz, float ks, T dx, float beta, float mu, int M, int dk,
                                         Out &&out) {
    const T eps = p2 - mu;
    const T E = fd_exp(-beta * fd_abs(eps));
    const T phi = rcp_approx(1.0f + E);
    const T psi = E * phi;
    const auto pos = fd_gt0(dx);
    const T tau = beta * dx;
    const auto occ = fd_lt0(eps);
    const T tstar = fd_sel(occ, fd_sel(pos, tau - beta, tau), fd_sel(pos, tau, tau + beta));
    const T X = fd_sel(pos, T(-1.0f), T(1.0f)) * fd_exp(-eps * tstar) * phi;
    if (M == 0 && !dk) {
        out(0, X);
        return;
    }
    const int Mx = M + dk;
    T ph[FD_MAX_M + 1], ps[FD_MAX_M + 1], A[FD_MAX_M + 1], cf[FD_MAX_M + 1];
    const T g = fd_sel(occ, T(beta), T(-beta));
    ph[0] = 1.0f;
    ps[0] = psi;
    A[0] = 1.0f;
#pragma unroll
    for (int k = 0; k < FD_MAX_M; ++k) {
        if (k < Mx) {
            T s = 0.0f;
#pragma unroll
            for (int i = 0; i <= k; ++i) s = fd_fma(ph[i], ps[k - i], s);
            ph[k + 1] = g * s * inv_int(k + 1);
            ps[k + 1] = -phi * ph[k + 1];
            A[k + 1] = A[k] * tstar * inv_int(k + 1);
        }
    }
#pragma unroll
    for (int j = 0; j <= FD_MAX_M; ++j) {
        if (j <= Mx) {
            T s = 0.0f;
#pragma unroll
            for (int i = 0; i <= j; ++i) s = fd_fma(A[j - i], ph[i], s);
            cf[j] = X * s;
        }
    }
#pragma unroll
    for (int j = 0; j <= FD_MAX_M; ++j)
        if (j <= M) out(j, cf[j]);
    if (dk) {
        // d eps / d k_ext = 2 p . e_z ks; d/dk c_j = -(j + 1) c_(j+1) d eps / dk
        const T kz = -2.0f * ks * pz;
#pragma unroll
        for (int j = 0; j < FD_MAX_M; ++j)
            if (j <= M) out(M + 1 + j, kz * (float)(j + 1) * cf[j + 1]);
    }
}

// V Taylor family: c_l = (d/dLambda)^l V / l! = 8 pi (-1)^l w^(l+1), w = 1/(q^2+Lambda),
// l <= L, then (when dk) d c_l / d k_ext.  out(l, value) receives (L + 1) (1 + dk) values.
template <class T, class Out>
__device__ __forceinline__ void v_family(T q2, T qz, float ks, float Lambda, int L, int dk, Out &&out) {
    const T inv = rcp_approx(q2 + Lambda);
    T cl = FD_8PI * inv;
    T cf[FD_MAX_M + 1];
#pragma unroll
    for (int l = 0; l <= FD_MAX_M; ++l) {
        if (l <= L + dk) {
            cf[l] = cl;
            cl = -inv * cl;
        }
    }
#pragma unroll
    for (int l = 0; l <= FD_MAX_M; ++l)
        if (l <= L) out(l, cf[l]);
    if (dk) {
        const T kz = 2.0f * ks * qz;
#pragma unroll
        for (int l = 0; l < FD_MAX_M; ++l)
            if (l <= L) out(L + 1 + l, kz * (float)(l + 1) * cf[l + 1]);
    }
}

// Out-of-line leaf families for the specialised kernels: one function per
// (M, dk) shape, called from every leaf of that shape, so the leaf code is
// fetched once and reused from the instruction cache instead of being inlined
// hundreds of times into straight-line code.
template <int NV>
struct FdLeafOut {
    float v[NV];
};

template <int M, int DK>
__device__ __noinline__ FdLeafOut<(M + 1) * (1 + DK)> g_leaf_fn(float p2, float pz, float ks, float dx, float beta,
                                                                 float mu) {
    FdLeafOut<(M + 1) * (1 + DK)> o;
    g_family(p2, pz, ks, dx, beta, mu, M, DK, [&](int j, float v) { o.v[j] = v; });
    return o;
}

template <int L, int DK>
__device__ __noinline__ FdLeafOut<(L + 1) * (1 + DK)> v_leaf_fn(float q2, float qz, float ks, float Lambda) {
    FdLeafOut<(L + 1) * (1 + DK)> o;
    v_family(q2, qz, ks, Lambda, L, DK, [&](int j, float v) { o.v[j] = v; });
    return o;
}

// ---- specialised kernels -------------------------------------------------------
// Per-sample variables the generated code reads: loop momenta k_1..k_N,
// hypercube times of the interaction lines (t[0] = 0) and the parameters.
template <class T>
struct FdSVT {
    T kx[FD_MAX_ORDER], ky[FD_MAX_ORDER], kz[FD_MAX_ORDER], t[FD_MAX_ORDER];
    float kext, beta, mu, Lam;
    float pad;                 // 29 words for float: an odd stride, so [sample][thread] rows in shared memory are conflict-free
};
using FdSV = FdSVT<float>;

// two samples' variables for the packed code (the parameters are per instance)
__device__ __forceinline__ FdSVT<FdF2> fd_pack(const FdSV &a, const FdSV &b) {
    FdSVT<FdF2> w;
#pragma unroll
    for (int j = 0; j < FD_MAX_ORDER; ++j) {
        w.kx[j] = FdF2(a.kx[j], b.kx[j]);
        w.ky[j] = FdF2(a.ky[j], b.ky[j]);
        w.kz[j] = FdF2(a.kz[j], b.kz[j]);
        w.t[j] = FdF2(a.t[j], b.t[j]);
    }
    w.kext = a.kext;
    w.beta = a.beta;
    w.mu = a.mu;
    w.Lam = a.Lam;
    return w;
}

// Hypercube point of sample i (Philox stream or given point), VEGAS map (when
// the instance has one), then loop momenta k_j, interaction-line times t_j
// (hypercube units, t_0 = 0) and the weight jac[n - 1] of the roots of order
// n (Jacobians of the roots' own coordinates, times the point weight).
// bins[d] receives the VEGAS bin of coordinate d (histogram).
// Layout: k_1 <- x[0:3]; k_j <- x[4j-5 : 4j-2] and the time of line j - 1 <- x[4j-2] for j >= 2.
template <int N, int DIM>
__device__ __forceinline__ void sample_point(const InstDesc &D, const EvalArgs &A, int64_t i, uint32_t iter,
                                             FdSV &V, float (&jac)[N], int (&bins)[DIM]) {
    float x[DIM];
    float wgt = 1.0f;
    if (D.points) {
#pragma unroll
        for (int d = 0; d < DIM; ++d) x[d] = D.points[(int64_t)d * A.n_per_inst + i];
        wgt = D.point_w ? D.point_w[i] : 1.0f;
    } else {
        const uint32_t c0 = (uint32_t)(uint64_t)i, c1 = (uint32_t)((uint64_t)i >> 32);
#pragma unroll
        for (int blk = 0; blk < (DIM + 3) / 4; ++blk) {
            const u32x4 r = philox4x32_10(u32x4{c0, c1, iter, ((uint32_t)D.id << 8) | (uint32_t)blk}, A.seed_lo,
                                          A.seed_hi);
            const uint32_t wv[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (4 * blk + q < DIM) x[4 * blk + q] = word_to_uniform(wv[q]);
        }
    }
    float jd[DIM];
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
        jd[d] = 1.0f;
        bins[d] = 0;
        if (D.edges) {
            const int nb = D.n_bins;
            const float y = x[d] * (float)nb;
            const int bin = min((int)y, nb - 1);
            const float *e = D.edges + (int64_t)d * (nb + 1);
            const float lo = __ldg(e + bin), hi = __ldg(e + bin + 1);
            x[d] = fmaf(y - (float)bin, hi - lo, lo);
            jd[d] = (float)nb * (hi - lo);
            bins[d] = bin;
        }
    }
    float w = wgt;
#pragma unroll
    for (int j = 0; j < N; ++j) {
        const int c0 = (j == 0) ? 0 : 4 * j - 1;
        const float xa = x[c0], xb = x[c0 + 1], xc = x[c0 + 2];
        const float r = D.kc * xa;
        const float cth = fmaf(2.0f, xb, -1.0f);
        const float sth = 2.0f * sqrtf(xb * (1.0f - xb));
        float sp, cp;
        sincospif(2.0f * xc, &sp, &cp);
        V.kx[j] = r * sth * cp;
        V.ky[j] = r * sth * sp;
        V.kz[j] = r * cth;
        w *= D.kc * r * r * FD_INV_2PI2;
        w *= jd[c0] * jd[c0 + 1] * jd[c0 + 2];
        V.t[j] = 0.0f;
        if (j >= 1) {
            V.t[j] = x[4 * j + 2];
            w *= D.beta * jd[4 * j + 2];
        }
        jac[j] = w;
    }
    V.kext = D.kext;
    V.beta = D.beta;
    V.mu = D.mu;
    V.Lam = D.Lambda;
}

// Completed roots of one sample: weight, optional per-sample output, warp
// reduction of (f, f^2) for the real and imaginary parts, and FP64 Neumaier
// accumulation per warp (lane 0).
template <int N>
struct FdSink {
    double *acc;                 // this warp's accumulators [R][4][2]
    const float *jac;            // [N]
    bool valid;
    float hsum;                  // sum over value roots of |Re f| + |Im f| (VEGAS histogram)
    float *ps;                   // per-sample output or null
    int64_t ps_row, ps_n;        // offset of (root 0, real part) and the row length

    template <int R_IDX, int ORD, int DK>
    __device__ __forceinline__ void flush(float re, float im) {
        const float J = jac[ORD - 1];
        const float fre = valid ? re * J : 0.0f;
        const float fim = valid ? im * J : 0.0f;
        if (!DK) hsum += fabsf(fre) + fabsf(fim);
        if (ps && valid) {
            ps[ps_row + (int64_t)(2 * R_IDX) * ps_n] = fre;
            ps[ps_row + (int64_t)(2 * R_IDX + 1) * ps_n] = fim;
        }
        float v[4] = {fre, fre * fre, fim, fim * fim};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], off);
        }
        if ((threadIdx.x & 31) == 0) {
#pragma unroll
            for (int q = 0; q < 4; ++q) neumaier(acc[(R_IDX * 4 + q) * 2], acc[(R_IDX * 4 + q) * 2 + 1], (double)v[q]);
        }
    }
};

// Completed root R_IDX for the P samples of this thread: per-sample weights,
// VEGAS sums and outputs, then one warp reduction of the thread's FP32 sums
// over its samples and one FP64 accumulation per warp (instead of one per sample).
template <int R_IDX, int ORD, int DK, int P, int N>
__device__ __forceinline__ void flush_samples(FdSink<N> *K, const float *re, const float *im) {
    float v[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const float J = K[p].jac[ORD - 1];
        const float fre = K[p].valid ? re[p] * J : 0.0f;
        const float fim = K[p].valid ? im[p] * J : 0.0f;
        if (!DK) K[p].hsum += fabsf(fre) + fabsf(fim);
        if (K[p].ps && K[p].valid) {
            K[p].ps[K[p].ps_row + (int64_t)(2 * R_IDX) * K[p].ps_n] = fre;
            K[p].ps[K[p].ps_row + (int64_t)(2 * R_IDX + 1) * K[p].ps_n] = fim;
        }
        v[0] += fre;
        v[1] = fmaf(fre, fre, v[1]);
        v[2] += fim;
        v[3] = fmaf(fim, fim, v[3]);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], off);
    }
    if ((threadIdx.x & 31) == 0) {
        double *acc = K[0].acc;
#pragma unroll
        for (int q = 0; q < 4; ++q) neumaier(acc[(R_IDX * 4 + q) * 2], acc[(R_IDX * 4 + q) * 2 + 1], (double)v[q]);
    }
}

// VEGAS histogram of one tile.  With hist_smem > 0 the launch provides
// dim x n_bins floats of dynamic shared memory: each sample adds its squared
// |f| sum to its bins there (FP32 shared atomics) and the tile's nonzero bins
// go to the FP64 global histogram once at the end of the tile, instead of one
// FP64 global atomic per sample and coordinate.  A square that overflows FP32
// goes straight to the global histogram.
template <int DIM>
__device__ __forceinline__ void hist_sample(const InstDesc &D, float *hs, const int *bins, float hsum) {
    const float h = hsum * hsum;
    if (hs && h <= 3.40282347e38f) {      // finite in FP32
#pragma unroll
        for (int d = 0; d < DIM; ++d) atomicAdd(hs + d * D.n_bins + bins[d], h);
    } else {
        const double hd = (double)hsum * (double)hsum;
#pragma unroll
        for (int d = 0; d < DIM; ++d) atomicAdd(D.hist + (int64_t)d * D.n_bins + bins[d], hd);
    }
}

template <int DIM, int T>
__device__ __forceinline__ void hist_tile_flush(const InstDesc &D, const float *hs) {
    for (int k = threadIdx.x; k < DIM * D.n_bins; k += T) {
        const float v = hs[k];
        if (v != 0.0f) atomicAdd(D.hist + k, (double)v);
    }
}

template <int DIM, int T>
__device__ __forceinline__ float *hist_tile_begin(const InstDesc &D, const EvalArgs &A, float *smem) {
    if (!D.hist || A.hist_smem < DIM * D.n_bins) return nullptr;
    for (int k = threadIdx.x; k < DIM * D.n_bins; k += T) smem[k] = 0.0f;
    __syncthreads();
    return smem;
}

// Persistent specialised kernel body: work items (instance, tile) from the
// queue, one sample per thread per pass, Body::run contracts the graph, tile
// partials combined over warps in a fixed order (bitwise reproducible).
template <class Body, int N, int DIM, int R, int T>
__device__ __forceinline__ void jit_main(const EvalArgs &A) {
    __shared__ double acc[T / 32][R * 8];
    __shared__ int next_item;
    extern __shared__ float hist_smem[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int n_items = A.n_inst * A.tiles_per_inst;
    const uint32_t iter = A.iter + (A.iter_dev ? *A.iter_dev : 0u);
    for (;;) {
        if (tid == 0) next_item = (int)atomicAdd(A.queue, 1ull);
        __syncthreads();
        const int item = next_item;
        if (item >= n_items) break;
        const InstDesc &D = A.inst[A.perm[item / A.tiles_per_inst]];
        const int tile = item % A.tiles_per_inst;
        for (int k = lane; k < R * 8; k += 32) acc[warp][k] = 0.0;
        __syncwarp();
        float *hs = hist_tile_begin<DIM, T>(D, A, hist_smem);
        const int64_t first = (int64_t)tile * A.tile;
        const int64_t last = min(first + A.tile, A.n_per_inst);
        for (int64_t base = first; base < last; base += T) {
            const int64_t i = base + tid;
            const bool valid = i < last;
            const int64_t idx = valid ? i : first;
            FdSV V;
            float jac[N];
            int bins[DIM];
            sample_point<N, DIM>(D, A, idx, iter, V, jac, bins);
            float cs[N], sn[N];
            cs[0] = 1.0f;
            sn[0] = 0.0f;
#pragma unroll
            for (int j = 1; j < N; ++j) sincospif(V.t[j], &sn[j], &cs[j]);   // exp(i pi x_line)
            FdSink<N> K{acc[warp], jac, valid, 0.0f, A.per_sample_f,
                        (int64_t)D.id * A.r_max * 2 * A.n_per_inst + idx, A.n_per_inst};
            Body::run(V, cs, sn, K);
            if (D.hist && valid) hist_sample<DIM>(D, hs, bins, K.hsum);
        }
        __syncthreads();
        if (hs) hist_tile_flush<DIM, T>(D, hs);
        for (int k = tid; k < R * 4; k += T) {
            double s = 0.0, c = 0.0;
            for (int wp = 0; wp < T / 32; ++wp) {
                neumaier(s, c, acc[wp][k * 2]);
                neumaier(s, c, acc[wp][k * 2 + 1]);
            }
            const int64_t o = (((int64_t)D.id * A.tiles_per_inst + tile) * A.r_max) * 4;
            A.partials[o + k] = s + c;     // k = r * 4 + q, q: re sum, re sumsq, im sum, im sumsq
        }
        for (int k = R * 4 + tid; k < A.r_max * 4; k += T) {
            const int64_t o = (((int64_t)D.id * A.tiles_per_inst + tile) * A.r_max) * 4;
            A.partials[o + k] = 0.0;
        }
        __syncthreads();
    }
}

// Variant with P samples per thread per pass, handled one after another by
// every compilation unit (Body::run loops over the samples inside each unit):
// the unit's code is fetched once and then re-executed from the instruction
// cache for the other P - 1 samples, at no cost in registers.  The per-sample
// inputs live in local memory (SVS = 1) or, with SVS = T, in dynamic shared
// memory as [sample][thread] rows of FdSV (sample p of this thread at
// V[p * SVS]); the tile histogram, when the launch provides it, follows them.
template <class Body, int N, int DIM, int R, int T, int P, int SVS = 1>
__device__ __forceinline__ void jit_main_loop(const EvalArgs &A) {
    __shared__ double acc[T / 32][R * 8];
    __shared__ int next_item;
    extern __shared__ float dyn_smem[];
    constexpr int SV_FLOATS = SVS > 1 ? T * P * (int)(sizeof(FdSV) / sizeof(float)) : 0;
    float *const hist_smem = dyn_smem + SV_FLOATS;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int n_items = A.n_inst * A.tiles_per_inst;
    const uint32_t iter = A.iter + (A.iter_dev ? *A.iter_dev : 0u);
    for (;;) {
        if (tid == 0) next_item = (int)atomicAdd(A.queue, 1ull);
        __syncthreads();
        const int item = next_item;
        if (item >= n_items) break;
        const InstDesc &D = A.inst[A.perm[item / A.tiles_per_inst]];
        const int tile = item % A.tiles_per_inst;
        for (int k = lane; k < R * 8; k += 32) acc[warp][k] = 0.0;
        __syncwarp();
        float *hs = hist_tile_begin<DIM, T>(D, A, hist_smem);
        const int64_t first = (int64_t)tile * A.tile;
        const int64_t last = min(first + A.tile, A.n_per_inst);
        for (int64_t base = first; base < last; base += (int64_t)T * P) {
            FdSV Vl[SVS > 1 ? 1 : P];
            FdSV *const V = SVS > 1 ? reinterpret_cast<FdSV *>(dyn_smem) + tid : Vl;
            float jac[P][N];
            int bins[P][DIM];
            float cs[P * N], sn[P * N];
            FdSink<N> K[P];
#pragma unroll
            for (int p = 0; p < P; ++p) {
                const int64_t i = base + (int64_t)p * T + tid;
                const bool valid = i < last;
                const int64_t idx = valid ? i : first;
                sample_point<N, DIM>(D, A, idx, iter, V[p * SVS], jac[p], bins[p]);
                cs[p * N] = 1.0f;
                sn[p * N] = 0.0f;
#pragma unroll
                for (int j = 1; j < N; ++j) sincospif(V[p * SVS].t[j], &sn[p * N + j], &cs[p * N + j]);
                K[p] = FdSink<N>{acc[warp], jac[p], valid, 0.0f, A.per_sample_f,
                                 (int64_t)D.id * A.r_max * 2 * A.n_per_inst + idx, A.n_per_inst};
            }
            Body::run(V, cs, sn, K);
            if (D.hist) {
#pragma unroll
                for (int p = 0; p < P; ++p)
                    if (K[p].valid) hist_sample<DIM>(D, hs, bins[p], K[p].hsum);
            }
        }
        __syncthreads();
        if (hs) hist_tile_flush<DIM, T>(D, hs);
        for (int k = tid; k < R * 4; k += T) {
            double s = 0.0, c = 0.0;
            for (int wp = 0; wp < T / 32; ++wp) {
                neumaier(s, c, acc[wp][k * 2]);
                neumaier(s, c, acc[wp][k * 2 + 1]);
            }
            const int64_t o = (((int64_t)D.id * A.tiles_per_inst + tile) * A.r_max) * 4;
            A.partials[o + k] = s + c;
        }
        for (int k = R * 4 + tid; k < A.r_max * 4; k += T) {
            const int64_t o = (((int64_t)D.id * A.tiles_per_inst + tile) * A.r_max) * 4;
            A.partials[o + k] = 0.0;
        }
        __syncthreads();
    }
}
