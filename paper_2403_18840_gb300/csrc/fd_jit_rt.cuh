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
#include <math.h>
#include <stdint.h>
#endif

// Functions marked FD_HD are plain FP32/FP64 arithmetic: the kernels call
// them, and a host build of this header runs the same code on the CPU.
#define FD_HD __host__ __device__ __forceinline__

// rounded sum and product that the compiler may not fuse into an FMA (the
// error-free transformations below depend on the rounding of each step)
FD_HD float fd_add_rn(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fadd_rn(a, b);
#else
    return a + b;
#endif
}
FD_HD float fd_mul_rn(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fmul_rn(a, b);
#else
    return a * b;
#endif
}

constexpr int FD_MAX_ORDER = 6;
constexpr int FD_MAX_DIM = 4 * FD_MAX_ORDER - 1;
constexpr int FD_MAX_M = 7;         // largest Taylor order of a leaf family (incl. d/dk)
constexpr int FD_LEAF_PRECISE_BIT = 44;   // G leaf word: evaluate the family in double-float (g_family_df)
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
    // k_ext and mu as grid parts (multiples of g and g^2), beta and K_c rounded
    // to FP32; with the remainders below they carry the FP64 parameters
    float kext, mu, beta, Lambda, kc;
    float kext_l, mu_l, beta_l, kc_l;
    float grid;                // g: a power of two, the grid of the loop-momentum components
    int32_t id;                // instance index of the call (partials, per-sample rows, Philox stream)
};

struct FdTab4;

struct EvalArgs {
    int32_t n_inst, tiles_per_inst, r_max, slots_total, dim_max;
    int32_t hist_smem;                 // floats of dynamic shared memory for the tile histogram (0: none)
    int64_t n_per_inst, tile;
    uint32_t seed_lo, seed_hi, iter;
    uint32_t wait_polls;               // tape waits of the interpreter give up after this many polls
    const uint32_t *iter_dev;          // optional: iteration += *iter_dev (read on the device)
    unsigned long long *queue;         // work counter (reset to 0 before the launch)
    double *partials;
    float *per_sample_f;
    float *abs_f;                      // optional [inst][n]: sum over value roots of |Re| + |Im| (0 if not finite)
    float *lc_global;                  // global leaf cache (one region of T x P x LCW floats per CTA) or null
    int *status;
    const FdTab4 *sc_tab;              // cos / sin of 2 pi n / 256 as double-float pairs, n = 0..256
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

// ---- accurate kinematics (double-float arithmetic in FP32) ------------------------
// A G0 coefficient of Eq. taylor_node depends on eps = |p|^2 - mu through
// exp(-eps tau*) and the Fermi factor; near the Fermi surface eps is a small
// difference of O(mu) numbers, and a derivative coefficient (d/dmu)^j G0 can
// vanish there (the equal-time line: f''(0) = 0).  Momenta rounded to FP32
// move eps by ~1e-6 and the coefficient by that much relative to its scale,
// so the sampler map, the loop momenta and eps are computed as unevaluated
// sums hi + lo of FP32 numbers (error-free transformations: Knuth's TwoSum,
// Dekker's product through an FMA) and eps is rounded to FP32 only at the end.
// Each loop-momentum component is stored as a "grid" part, a multiple of the
// instance's power of two g (so that the signed momentum sums of a leaf, and
// their squares near the Fermi surface, are exact in FP32), plus a small
// remainder |lo| <= g/2 carried in FP32.
struct FdDF {
    float hi, lo;
};

FD_HD FdDF fd_two_sum(float a, float b) {
    const float s = fd_add_rn(a, b);
    const float bb = fd_add_rn(s, -a);
    const float e = fd_add_rn(fd_add_rn(a, -fd_add_rn(s, -bb)), fd_add_rn(b, -bb));
    return FdDF{s, e};
}
// |a| >= |b| (or a == 0)
FD_HD FdDF fd_fast_two_sum(float a, float b) {
    const float s = fd_add_rn(a, b);
    return FdDF{s, fd_add_rn(b, -fd_add_rn(s, -a))};
}
FD_HD FdDF fd_two_prod(float a, float b) {
    const float p = fd_mul_rn(a, b);
    return FdDF{p, fmaf(a, b, -p)};
}
FD_HD FdDF fd_df_mul(FdDF a, FdDF b) {
    const FdDF p = fd_two_prod(a.hi, b.hi);
    return fd_fast_two_sum(p.hi, p.lo + fmaf(a.hi, b.lo, a.lo * b.hi));
}
// a b for an FP32 b
FD_HD FdDF fd_df_mulf(FdDF a, float b) {
    const FdDF p = fd_two_prod(a.hi, b);
    return fd_fast_two_sum(p.hi, fmaf(a.lo, b, p.lo));
}
// a + b: the error is a few 2^-48 of |a| + |b| (enough where a sum cancels
// to ~1e-9 of its terms and keeps 1e-5 of its own value)
FD_HD FdDF fd_df_add(FdDF a, FdDF b) {
    const FdDF s = fd_two_sum(a.hi, b.hi);
    return fd_two_sum(s.hi, fd_add_rn(s.lo, fd_add_rn(a.lo, b.lo)));
}
FD_HD FdDF fd_df_addf(FdDF a, float b) {
    const FdDF s = fd_two_sum(a.hi, b);
    return fd_two_sum(s.hi, fd_add_rn(s.lo, a.lo));
}
FD_HD FdDF fd_df_neg(FdDF a) { return FdDF{-a.hi, -a.lo}; }

// 1 / d for d in [1, 2]: the rounded FP32 reciprocal r and one Newton step
// r + r (1 - d r), with 1 - d r from the exact product d.hi r
FD_HD FdDF fd_df_rcp(FdDF d) {
#ifdef __CUDA_ARCH__
    const float r = __frcp_rn(d.hi);
#else
    const float r = 1.0f / d.hi;
#endif
    const FdDF p = fd_two_prod(d.hi, r);
    const float e = fd_add_rn(fd_add_rn(fd_add_rn(1.0f, -p.hi), -p.lo), -fd_mul_rn(d.lo, r));   // 1 - p.hi exact
    return fd_fast_two_sum(r, fd_mul_rn(r, e));
}

// 2^k as FP32 for -126 <= k <= 127
FD_HD float fd_pow2i(int k) {
#ifdef __CUDA_ARCH__
    return __int_as_float((k + 127) << 23);
#else
    return ldexpf(1.0f, k);
#endif
}

// exp(y) for y = y.hi + y.lo <= 0 as a double-float: relative error ~1e-15
// while exp(y) >= 2^-100 (y >= -69; its low part is then a normal FP32
// number), growing to the FP32 rounding (2^-24) as the low part runs into the
// subnormals near 2^-126; 0 for y <= -103, where exp(y) < 2^-148.  Cody and Waite's reduction y = n ln2 + r, |r| <= ln2 / 2,
// with ln2 = L1 + L2 + L3 (L1 has 15 significant bits, so n L1 is exact for
// |n| < 512); exp(r) = (1 + m)^16 with m = expm1(r / 16) from its Taylor
// series (|r / 16| < 0.022: the terms from the fifth on in FP32, the series
// ends at the seventh) and 16 = 2^4 squarings (1 + m)^2 = 1 + m (2 + m), which
// keep m's relative precision; then 2^n as two exact power-of-two factors.
FD_HD FdDF fd_exp_df(FdDF y) {
    if (!(y.hi > -103.0f)) return FdDF{0.0f, 0.0f};
    const float L1 = 0x1.62e4p-1f, L2 = 0x1.7f7d1cp-20f, L3 = 0x1.ef357ap-45f;
    const float n = rintf(fd_mul_rn(y.hi, 0x1.715476p+0f));
    FdDF r = fd_two_sum(y.hi, -fd_mul_rn(n, L1));
    r = fd_df_add(r, fd_df_neg(fd_two_prod(n, L2)));
    r = fd_df_add(r, fd_two_sum(y.lo, -fd_mul_rn(n, L3)));
    const FdDF h = FdDF{fd_mul_rn(r.hi, 0.0625f), fd_mul_rn(r.lo, 0.0625f)};
    // m = h (1 + h (1/2 + h (1/6 + h (1/24 + h t)))), t = 1/120 + h/720 + h^2/5040
    const float t = fmaf(h.hi, fmaf(h.hi, 1.0f / 5040.0f, 1.0f / 720.0f), 1.0f / 120.0f);
    FdDF p = fd_df_add(FdDF{0x1.555556p-5f, -0x1.555556p-30f}, fd_df_mulf(h, t));   // 1/24 + h t
    p = fd_df_add(FdDF{0x1.555556p-3f, -0x1.555556p-28f}, fd_df_mul(h, p));         // 1/6 + h p
    p = fd_df_addf(fd_df_mul(h, p), 0.5f);
    p = fd_df_addf(fd_df_mul(h, p), 1.0f);
    FdDF m = fd_df_mul(h, p);
#pragma unroll
    for (int i = 0; i < 4; ++i) m = fd_df_mul(m, fd_df_addf(m, 2.0f));
    const FdDF e = fd_df_addf(m, 1.0f);
    const int ni = (int)n, n1 = ni / 2;   // -149 <= n <= 0: both factors normal
    const float s1 = fd_pow2i(n1), s2 = fd_pow2i(ni - n1);
    return FdDF{fd_mul_rn(fd_mul_rn(e.hi, s1), s2), fd_mul_rn(fd_mul_rn(e.lo, s1), s2)};
}

// 1 / k as a double-float pair, k = 1..8
FD_HD FdDF fd_df_inv_int(int k) {
    return k == 1 ? FdDF{1.0f, 0.0f} : k == 2 ? FdDF{0.5f, 0.0f}
         : k == 3 ? FdDF{0x1.555556p-2f, -0x1.555556p-27f} : k == 4 ? FdDF{0.25f, 0.0f}
         : k == 5 ? FdDF{0x1.99999ap-3f, -0x1.99999ap-29f} : k == 6 ? FdDF{0x1.555556p-3f, -0x1.555556p-28f}
         : k == 7 ? FdDF{0x1.24924ap-3f, -0x1.b6db6ep-28f} : FdDF{0.125f, 0.0f};
}

// cos(2 pi c), sin(2 pi c) for c = c.hi + c.lo in [0, 1], relative accuracy
// ~1e-13.  tab[n] = (cos hi, cos lo, sin hi, sin lo) of 2 pi n / 256,
// n = 0..256, as double-float pairs; the remainder angle b = 2 pi (c - n/256),
// |b| <= pi/256, enters through sin b = b (1 - b^2/6 + b^4/120) and
// cos b = 1 + d, d = -b^2/2 + b^4/24 (the next terms are below 1e-14).
struct FdTab4 {
    float x, y, z, w;
};

FD_HD void fd_sincos2pi_df(FdDF c, const FdTab4 *tab, FdDF &cs, FdDF &sn) {
    const float n = rintf(c.hi * 256.0f);
    const float rh = fd_add_rn(c.hi, -n * 0.00390625f);          // exact (Sterbenz)
    const float kH = 6.28318548202514648f, kL = -1.7484555314695172e-07f;   // 2 pi = kH + kL
    const FdDF bp = fd_two_prod(kH, rh);
    const FdDF b = fd_fast_two_sum(bp.hi, bp.lo + fmaf(kH, c.lo, kL * rh));
    const float u = b.hi * b.hi;
    const float sb_hi = b.hi;
    const float sb_lo = fmaf(b.hi, u * fmaf(u, 1.0f / 120.0f, -1.0f / 6.0f), b.lo);
    const FdDF q = fd_two_prod(b.hi, b.hi);
    const float d_hi = -0.5f * q.hi;                                // exact
    const float d_lo = fmaf(q.hi * q.hi, 1.0f / 24.0f, -0.5f * fmaf(2.0f * b.hi, b.lo, q.lo));
    const FdTab4 t = tab[(int)n];
    // cos(a + b) = ca + ca d - sa sin b
    {
        const FdDF p1 = fd_two_prod(t.x, d_hi), p2 = fd_two_prod(t.z, sb_hi);
        const float rest = t.y + fmaf(t.x, d_lo, t.y * d_hi) + p1.lo - p2.lo - fmaf(t.z, sb_lo, t.w * sb_hi);
        const FdDF x = fd_two_sum(p1.hi, -p2.hi);
        const FdDF y = fd_two_sum(t.x, x.hi);
        cs = fd_two_sum(y.hi, y.lo + x.lo + rest);
    }
    // sin(a + b) = sa + sa d + ca sin b
    {
        const FdDF p3 = fd_two_prod(t.z, d_hi), p4 = fd_two_prod(t.x, sb_hi);
        const float rest = t.w + fmaf(t.z, d_lo, t.w * d_hi) + p3.lo + p4.lo + fmaf(t.x, sb_lo, t.y * sb_hi);
        const FdDF x = fd_two_sum(p3.hi, p4.hi);
        const FdDF y = fd_two_sum(t.z, x.hi);
        sn = fd_two_sum(y.hi, y.lo + x.lo + rest);
    }
}

// VEGAS map of one coordinate (Lepage): y = u nb, bin i = floor(y),
// x = e_i + (y - i) (e_(i+1) - e_i) from the FP32 edges, as hi + lo; returns
// the bin and the map's Jacobian nb (e_(i+1) - e_i).
FD_HD int fd_vegas_df(float u, int nb, const float *e, FdDF &x, float &jd) {
    const FdDF y = fd_two_prod(u, (float)nb);                       // y.lo = 0 for a power-of-two nb
    int bin = (int)y.hi;
    float fh = y.hi - (float)bin;                                   // exact
    if (fh == 0.0f && y.lo < 0.0f && bin > 0) {                     // just below the integer y.hi
        bin -= 1;
        fh = 1.0f;
    }
    if (bin > nb - 1) {                                             // u rounded up to 1: last bin
        bin = nb - 1;
        fh = 1.0f;
    }
    const float lo = e[bin], hi = e[bin + 1];
    const FdDF w = fd_two_sum(hi, -lo);
    const FdDF t = fd_two_prod(fh, w.hi);
    const FdDF s = fd_two_sum(lo, t.hi);
    x = fd_fast_two_sum(s.hi, s.lo + fmaf(fh, w.lo, fmaf(y.lo, w.hi, t.lo)));
    jd = (float)nb * w.hi;
    return bin;
}

// grid part and remainder of a double-float number: v = hi + lo with hi a
// multiple of g (g, ginv powers of two)
FD_HD void fd_grid_split(FdDF v, float g, float ginv, float &hi, float &lo) {
    hi = rintf(v.hi * ginv) * g;
    lo = fd_add_rn(v.hi, -hi) + v.lo;                               // v.hi - hi exact
}

// Loop momentum from its three hypercube coordinates (Sec. IV, spherical
// coordinates with cutoff K_c): r = K_c a, cos(theta) = 2 b - 1,
// sin(theta) = 2 sqrt(b (1 - b)), phi = 2 pi c; components split onto the
// grid g.  kc = K_c as hi + lo.  Returns r (FP32) for the Jacobian.
FD_HD float fd_loop_momentum(FdDF a, FdDF b, FdDF c, FdDF kc, const FdTab4 *tab, float g, float ginv,
                             float (&kh)[3], float (&kl)[3]) {
    const FdDF rp = fd_two_prod(kc.hi, a.hi);
    const FdDF r = FdDF{rp.hi, rp.lo + fmaf(kc.hi, a.lo, kc.lo * a.hi)};
    const FdDF c2 = fd_two_sum(2.0f * b.hi, -1.0f);
    const FdDF cth = FdDF{c2.hi, fmaf(2.0f, b.lo, c2.lo)};
    const FdDF om = fd_two_sum(1.0f, -b.hi);
    const FdDF wp = fd_two_prod(b.hi, om.hi);
    const float w_lo = wp.lo + fmaf(b.hi, om.lo - b.lo, b.lo * om.hi);
    const float sq = sqrtf(wp.hi);
    const float sq_lo = sq > 0.0f ? (fmaf(-sq, sq, wp.hi) + w_lo) * (0.5f / sq) : 0.0f;   // b = 0 or 1: sin = 0
    const FdDF sth = FdDF{2.0f * sq, 2.0f * sq_lo};
    FdDF cp, sp;
    fd_sincos2pi_df(c, tab, cp, sp);
    const FdDF rs = fd_df_mul(r, sth);
    fd_grid_split(fd_df_mul(rs, cp), g, ginv, kh[0], kl[0]);
    fd_grid_split(fd_df_mul(rs, sp), g, ginv, kh[1], kl[1]);
    fd_grid_split(fd_df_mul(r, cth), g, ginv, kh[2], kl[2]);
    return r.hi;
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
FD_HD float rcp_approx(float x) {
#ifdef __CUDA_ARCH__
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
#else
    return 1.0f / x;
#endif
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
FD_HD float fd_fma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ FdF2 fd_fma(FdF2 a, FdF2 b, FdF2 c) { return fd_wrap(__ffma2_rn(a.v, b.v, c.v)); }
FD_HD float fd_abs(float a) { return fabsf(a); }
__device__ __forceinline__ FdF2 fd_abs(FdF2 a) { return FdF2(fabsf(a.v.x), fabsf(a.v.y)); }
FD_HD float fd_exp(float a) {
#ifdef __CUDA_ARCH__
    return __expf(a);
#else
    return expf(a);
#endif
}
__device__ __forceinline__ FdF2 fd_exp(FdF2 a) { return FdF2(__expf(a.v.x), __expf(a.v.y)); }
FD_HD bool fd_gt0(float a) { return a > 0.0f; }
__device__ __forceinline__ FdM2 fd_gt0(FdF2 a) { return FdM2{a.v.x > 0.0f, a.v.y > 0.0f}; }
FD_HD bool fd_lt0(float a) { return a < 0.0f; }
__device__ __forceinline__ FdM2 fd_lt0(FdF2 a) { return FdM2{a.v.x < 0.0f, a.v.y < 0.0f}; }
FD_HD float fd_sel(bool c, float a, float b) { return c ? a : b; }
__device__ __forceinline__ FdF2 fd_sel(FdM2 c, FdF2 a, FdF2 b) {
    return FdF2(c.x ? a.v.x : b.v.x, c.y ? a.v.y : b.v.y);
}
__device__ __forceinline__ FdF2 rcp_approx(FdF2 x) { return FdF2(rcp_approx(x.v.x), rcp_approx(x.v.y)); }

// 1 / (k + 1) for the Taylor recurrences (no division in the inner loops)
FD_HD float inv_int(int k1) {
    return k1 == 1 ? 1.0f : k1 == 2 ? 0.5f : k1 == 3 ? 0.33333334f : k1 == 4 ? 0.25f
         : k1 == 5 ? 0.2f : k1 == 6 ? 0.16666667f : k1 == 7 ? 0.14285715f : 0.125f;
}
template <class T>
FD_HD T fd_inv_int(int k1) {
    return T(inv_int(k1));
}

// eps = |p|^2 - mu from a leaf's grid sums (ph: exact in FP32) and remainder
// sums (pl): the grid part sum ph^2 - mu_h is exact near the Fermi surface
// (ph on the grid g, mu_h on the grid g^2), the rest
// sum (2 ph + pl) pl - mu_l is small and rounds at ~1e-10.
template <class T>
FD_HD T fd_eps(T pxh, T pyh, T pzh, T pxl, T pyl, T pzl, float muh, float mul) {
    const T s = fd_fma(pxh, pxh, fd_fma(pyh, pyh, pzh * pzh)) - T(muh);
    const T L = fd_fma(fd_fma(T(2.0f), pxh, pxl), pxl,
                       fd_fma(fd_fma(T(2.0f), pyh, pyl), pyl, fd_fma(fd_fma(T(2.0f), pzh, pzl), pzl, T(-mul))));
    return s + L;
}

// hypercube time difference t_a - t_b of two interaction lines as hi + lo,
// normalised so that hi == 0 only for equal times
template <class T>
FD_HD void fd_time_diff(T tah, T tal, T tbh, T tbl, T &dh, T &dl) {
    const T s = tah - tbh;
    const T bb = s - tah;
    const T e = (tah - (s - bb)) + ((T(0.0f) - tbh) - bb);
    const T lo = e + (tal - tbl);
    dh = s + lo;
    dl = lo - (dh - s);
}



// ---- leaf families (Eq. taylor_node) -------------------------------------------
// G0 Taylor family at eps = |p|^2 - mu (pz = p_z; ks = coefficient of k_ext in
// p) and hypercube time difference dx = dxh + dxl of its two interaction
// lines: c_j = (d/dmu)^j G0 / j!, j <= M, then (when dk) d c_j / d k_ext, j <= M.
// Written as sign * exp(-eps tau*) * phi(eps - dmu) with the Fermi factor
// phi >= 1/2 (phi = 1 - f for eps >= 0, f for eps < 0) and tau* = beta dx* the
// matching antiperiodic time, dx* = dx - 1, dx or dx + 1 (exact in FP32 for
// the dyadic times of the hypercube), so the exponent is never positive.  The
// series of phi(eps - d) follows from the logistic ODE
// d phi / d eps = +-beta phi (1 - phi) (a Taylor-mode recurrence); the series
// of exp(d tau*) is tau*^k / k!.  T = float or the packed FdF2 (the
// families whose value is the only term of a root: g_family_df).  out(j,
// value) receives the (M + 1) (1 + dk) values.
template <class T, class Out>
FD_HD void g_family(T eps, T pz, float ks, T dxh, T dxl, T beta, int M, int dk, Out &&out) {
    const T E = fd_exp(-beta * fd_abs(eps));
    const T phi = rcp_approx(T(1.0f) + E);
    const T psi = E * phi;
    const auto pos = fd_gt0(dxh);
    const auto occ = fd_lt0(eps);
    const T dstar = fd_sel(occ, fd_sel(pos, dxh - T(1.0f), dxh), fd_sel(pos, dxh, dxh + T(1.0f))) + dxl;
    const T tstar = beta * dstar;
    const T X = fd_sel(pos, T(-1.0f), T(1.0f)) * fd_exp(-eps * tstar) * phi;
    if (M == 0 && !dk) {
        out(0, X);
        return;
    }
    const int Mx = M + dk;
    T ph[FD_MAX_M + 1], ps[FD_MAX_M + 1], A[FD_MAX_M + 1], cf[FD_MAX_M + 1];
    const T g = fd_sel(occ, beta, T(0.0f) - beta);
    ph[0] = T(1.0f);
    ps[0] = psi;
    A[0] = T(1.0f);
#pragma unroll
    for (int k = 0; k < FD_MAX_M; ++k) {
        if (k < Mx) {
            T s = T(0.0f);
#pragma unroll
            for (int i = 0; i <= k; ++i) s = fd_fma(ph[i], ps[k - i], s);
            ph[k + 1] = g * s * fd_inv_int<T>(k + 1);
            ps[k + 1] = (T(0.0f) - phi) * ph[k + 1];
            A[k + 1] = A[k] * tstar * fd_inv_int<T>(k + 1);
        }
    }
#pragma unroll
    for (int j = 0; j <= FD_MAX_M; ++j) {
        if (j <= Mx) {
            T s = T(0.0f);
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
        const T kz = T(-2.0f * ks) * pz;
#pragma unroll
        for (int j = 0; j < FD_MAX_M; ++j)
            if (j <= M) out(M + 1 + j, kz * T((float)(j + 1)) * cf[j + 1]);
    }
}

// The G0 family of a line whose coefficients are, alone, the value of a root
// (the single line of the order-1 diagram): a coefficient (d/dmu)^j G0 of the
// equal-time line has zeros in eps (f''(0) = 0 and the nonzero roots of the
// higher logistic derivatives), near which an FP32 evaluation has a large
// error relative to the value itself.
// This family is therefore evaluated in double-float arithmetic (pairs of
// FP32 numbers, ~48 significant bits) rather than FP64, whose instructions
// issue at a small fraction of the FP32 rate on this GPU.  Inputs: the line's
// momentum as grid parts (ph) and double-float remainders (pl), the time
// difference dx = dxh + dxl, beta and mu as hi + lo.  eps = |ph + pl|^2 - mu
// from exact products; E = exp(-beta |eps|) (fd_exp_df), the Fermi factor
// phi = 1 / (1 + E) and psi = E phi, tau* = beta dx*, the Taylor recurrences of
// g_family and the coefficient sums in double-float; the common factor
// exp(-eps tau*) phi, which no sum cancels, in FP32 from the accurate expf of
// the product's high part times 1 - (its low part).
template <class Out>
FD_HD void g_family_df(float pxh, float pyh, float pzh, FdDF pxl, FdDF pyl, FdDF pzl, float ks, float dxh,
                       float dxl, float bh, float bl, float muh, float mul, int M, int dk, Out &&out) {
    // |ph + pl|^2 = sum ph^2 + 2 ph pl.hi + (2 ph pl.lo + pl.hi^2), the last
    // terms below 1e-7 and rounded once
    FdDF e2 = fd_two_prod(pxh, pxh);
    e2 = fd_df_add(e2, fd_two_prod(pyh, pyh));
    e2 = fd_df_add(e2, fd_two_prod(pzh, pzh));
    e2 = fd_df_addf(e2, -muh);
    FdDF cr = fd_two_prod(2.0f * pxh, pxl.hi);
    cr = fd_df_add(cr, fd_two_prod(2.0f * pyh, pyl.hi));
    cr = fd_df_add(cr, fd_two_prod(2.0f * pzh, pzl.hi));
    const float small = fmaf(2.0f * pxh, pxl.lo, fmaf(pxl.hi, pxl.hi, fmaf(2.0f * pyh, pyl.lo,
                        fmaf(pyl.hi, pyl.hi, fmaf(2.0f * pzh, pzl.lo, fmaf(pzl.hi, pzl.hi, -mul))))));
    const FdDF eps = fd_df_addf(fd_df_add(e2, cr), small);
    const bool occ = eps.hi < 0.0f;
    const FdDF beta = FdDF{bh, bl};
    const FdDF E = fd_exp_df(fd_df_neg(fd_df_mul(beta, occ ? fd_df_neg(eps) : eps)));
    const FdDF phi = fd_df_rcp(fd_df_addf(E, 1.0f));
    const FdDF psi = fd_df_mul(E, phi);
    const bool et = dxh == 0.0f && dxl == 0.0f;   // equal times (0^-): tau* = 0 or beta
    const bool pos = dxh > 0.0f;
    const float shift = occ ? (pos ? -1.0f : 0.0f) : (pos ? 0.0f : 1.0f);
    const FdDF tstar = fd_df_mul(beta, fd_df_addf(fd_two_sum(dxh, shift), dxl));
    float X;
    if (et) {
        X = occ ? phi.hi : psi.hi;
    } else {
        const FdDF y = fd_df_mul(eps, tstar);   // >= 0: the exponent -eps tau* is never positive
        X = (pos ? -1.0f : 1.0f) * fd_mul_rn(fd_mul_rn(expf(-y.hi), 1.0f - y.lo), phi.hi);
    }
    if (M == 0 && !dk) {
        out(0, X);
        return;
    }
    const int Mx = M + dk;
    const FdDF g = occ ? beta : fd_df_neg(beta);
    FdDF ph[FD_MAX_M + 1], ps[FD_MAX_M + 1], A[FD_MAX_M + 1];
    ph[0] = FdDF{1.0f, 0.0f};
    ps[0] = psi;
    A[0] = FdDF{1.0f, 0.0f};
#pragma unroll
    for (int k = 0; k < FD_MAX_M; ++k) {
        if (k < Mx) {
            FdDF s = ps[k];   // ph[0] = 1
#pragma unroll
            for (int i = 1; i <= k; ++i) s = fd_df_add(s, fd_df_mul(ph[i], ps[k - i]));
            const FdDF inv = fd_df_inv_int(k + 1);
            ph[k + 1] = fd_df_mul(fd_df_mul(g, s), inv);
            ps[k + 1] = fd_df_neg(fd_df_mul(phi, ph[k + 1]));
            A[k + 1] = fd_df_mul(fd_df_mul(A[k], tstar), inv);
        }
    }
    float cf[FD_MAX_M + 1];
#pragma unroll
    for (int j = 0; j <= FD_MAX_M; ++j) {
        if (j <= Mx) {
            FdDF s = fd_df_add(A[j], ph[j]);   // the terms i = 0 and i = j (j >= 1)
            if (j == 0) s = FdDF{1.0f, 0.0f};
#pragma unroll
            for (int i = 1; i < j; ++i) s = fd_df_add(s, fd_df_mul(A[j - i], ph[i]));
            cf[j] = fmaf(X, s.hi, X * s.lo);
        }
    }
#pragma unroll
    for (int j = 0; j <= FD_MAX_M; ++j)
        if (j <= M) out(j, cf[j]);
    if (dk) {
        const float kz = -2.0f * ks * (pzh + pzl.hi);
#pragma unroll
        for (int j = 0; j < FD_MAX_M; ++j)
            if (j <= M) out(M + 1 + j, kz * (float)(j + 1) * cf[j + 1]);
    }
}

// V Taylor family: c_l = (d/dLambda)^l V / l! = 8 pi (-1)^l w^(l+1), w = 1/(q^2+Lambda),
// l <= L, then (when dk) d c_l / d k_ext.  out(l, value) receives (L + 1) (1 + dk) values.
template <class T, class Out>
FD_HD void v_family(T q2, T qz, float ks, float Lambda, int L, int dk, Out &&out) {
    const T inv = rcp_approx(q2 + T(Lambda));
    T cl = T(FD_8PI) * inv;
    T cf[FD_MAX_M + 1];
#pragma unroll
    for (int l = 0; l <= FD_MAX_M; ++l) {
        if (l <= L + dk) {
            cf[l] = cl;
            cl = (T(0.0f) - inv) * cl;
        }
    }
#pragma unroll
    for (int l = 0; l <= FD_MAX_M; ++l)
        if (l <= L) out(l, cf[l]);
    if (dk) {
        const T kz = T(2.0f * ks) * qz;
#pragma unroll
        for (int l = 0; l < FD_MAX_M; ++l)
            if (l <= L) out(L + 1 + l, kz * T((float)(l + 1)) * cf[l + 1]);
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
__device__ __noinline__ FdLeafOut<(M + 1) * (1 + DK)> g_leaf_fn(float eps, float pz, float ks, float dxh, float dxl,
                                                                 float beta) {
    FdLeafOut<(M + 1) * (1 + DK)> o;
    g_family<float>(eps, pz, ks, dxh, dxl, beta, M, DK, [&](int j, float v) { o.v[j] = v; });
    return o;
}

template <int L, int DK>
__device__ __noinline__ FdLeafOut<(L + 1) * (1 + DK)> v_leaf_fn(float q2, float qz, float ks, float Lambda) {
    FdLeafOut<(L + 1) * (1 + DK)> o;
    v_family<float>(q2, qz, ks, Lambda, L, DK, [&](int j, float v) { o.v[j] = v; });
    return o;
}

// ---- specialised kernels -------------------------------------------------------
// Per-sample variables the generated code reads: loop momenta k_1..k_N as grid
// parts (kx, ky, kz) and remainders (kxl, kyl, kzl), hypercube times of the
// interaction lines (t[0] = 0) as hi + lo.  8 N + 1 words for float: an odd
// stride, so [sample][thread] rows in shared memory are conflict-free.
template <class T, int N>
struct FdSVT {
    T kx[N], ky[N], kz[N], kxl[N], kyl[N], kzl[N], t[N], tl[N];
    float pad;
};
__host__ __device__ constexpr int fd_sv_words(int N) { return 8 * N + 1; }

// Per-instance parameters of the generated code: k_ext and mu as grid part +
// remainder (grid g and g^2), beta (and its remainder for the
// double-float families), Lambda.
struct FdPar {
    float kexth, kextl, beta, betal, muh, mul, Lam;
};

__device__ __forceinline__ FdPar fd_par(const InstDesc &D) {
    return FdPar{D.kext, D.kext_l, D.beta, D.beta_l, D.mu, D.mu_l, D.Lambda};
}

// two samples' variables for the packed code
template <int N>
__device__ __forceinline__ FdSVT<FdF2, N> fd_pack(const FdSVT<float, N> &a, const FdSVT<float, N> &b) {
    FdSVT<FdF2, N> w;
#pragma unroll
    for (int j = 0; j < N; ++j) {
        w.kx[j] = FdF2(a.kx[j], b.kx[j]);
        w.ky[j] = FdF2(a.ky[j], b.ky[j]);
        w.kz[j] = FdF2(a.kz[j], b.kz[j]);
        w.kxl[j] = FdF2(a.kxl[j], b.kxl[j]);
        w.kyl[j] = FdF2(a.kyl[j], b.kyl[j]);
        w.kzl[j] = FdF2(a.kzl[j], b.kzl[j]);
        w.t[j] = FdF2(a.t[j], b.t[j]);
        w.tl[j] = FdF2(a.tl[j], b.tl[j]);
    }
    return w;
}


// Hypercube point of sample i (Philox stream or given point), VEGAS map (when
// the instance has one), then loop momenta k_j, interaction-line times t_j
// (hypercube units, t_0 = 0) and the weight jac[n - 1] of the roots of order
// n (Jacobians of the roots' own coordinates, times the point weight).
// bins[d] receives the VEGAS bin of coordinate d (histogram).  Mapped
// coordinates, momenta and times are double-float (hi + lo); the weights FP32.
// Layout: k_1 <- x[0:3]; k_j <- x[4j-5 : 4j-2] and the time of line j - 1 <- x[4j-2] for j >= 2.
template <int N, int DIM>
__device__ __forceinline__ void sample_point(const InstDesc &D, const EvalArgs &A, int64_t i, uint32_t iter,
                                             FdSVT<float, N> &V, float (&jac)[N], int (&bins)[DIM]) {
    FdDF x[DIM];
    float wgt = 1.0f;
    if (D.points) {
#pragma unroll
        for (int d = 0; d < DIM; ++d) x[d] = FdDF{D.points[(int64_t)d * A.n_per_inst + i], 0.0f};
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
                if (4 * blk + q < DIM) x[4 * blk + q] = FdDF{word_to_uniform(wv[q]), 0.0f};
        }
    }
    float jd[DIM];
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
        jd[d] = 1.0f;
        bins[d] = 0;
        if (D.edges) bins[d] = fd_vegas_df(x[d].hi, D.n_bins, D.edges + (int64_t)d * (D.n_bins + 1), x[d], jd[d]);
    }
    const float g = D.grid, ginv = 1.0f / D.grid;
    float w = wgt;
#pragma unroll
    for (int j = 0; j < N; ++j) {
        const int c0 = (j == 0) ? 0 : 4 * j - 1;
        float kh[3], kl[3];
        const float r = fd_loop_momentum(x[c0], x[c0 + 1], x[c0 + 2], FdDF{D.kc, D.kc_l}, A.sc_tab, g, ginv, kh, kl);
        V.kx[j] = kh[0];
        V.ky[j] = kh[1];
        V.kz[j] = kh[2];
        V.kxl[j] = kl[0];
        V.kyl[j] = kl[1];
        V.kzl[j] = kl[2];
        w *= D.kc * r * r * FD_INV_2PI2;
        w *= jd[c0] * jd[c0 + 1] * jd[c0 + 2];
        V.t[j] = 0.0f;
        V.tl[j] = 0.0f;
        if (j >= 1) {
            V.t[j] = x[4 * j + 2].hi;
            V.tl[j] = x[4 * j + 2].lo;
            w *= D.beta * jd[4 * j + 2];
        }
        jac[j] = w;
    }
}

// Completed roots of one sample: weight, optional per-sample output, warp
// reduction of (f, f^2) for the real and imaginary parts, and FP64 Neumaier
// accumulation per warp (lane 0).
// The four warp totals (Re f, (Re f)^2, Im f, (Im f)^2; every lane holds the
// same values after the xor butterfly) into the warp's FP64 Neumaier
// accumulators acc[q][2], one per lane 0..3, so that the four FP64 updates
// run side by side instead of one after another in lane 0.
__device__ __forceinline__ void fd_accumulate_lanes(double *acc, const float (&v)[4]) {
    const int q = threadIdx.x & 31;
    if (q < 4) {
        const float mine = q == 0 ? v[0] : q == 1 ? v[1] : q == 2 ? v[2] : v[3];
        neumaier(acc[2 * q], acc[2 * q + 1], (double)mine);
    }
}

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
        fd_accumulate_lanes(acc + R_IDX * 8, v);
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
    fd_accumulate_lanes(K[0].acc + R_IDX * 8, v);
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
        const FdPar Q = fd_par(D);
        for (int k = lane; k < R * 8; k += 32) acc[warp][k] = 0.0;
        __syncwarp();
        float *hs = hist_tile_begin<DIM, T>(D, A, hist_smem);
        const int64_t first = (int64_t)tile * A.tile;
        const int64_t last = min(first + A.tile, A.n_per_inst);
        for (int64_t base = first; base < last; base += T) {
            const int64_t i = base + tid;
            const bool valid = i < last;
            const int64_t idx = valid ? i : first;
            FdSVT<float, N> V;
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
            Body::run(V, Q, cs, sn, K);
            if (D.hist && valid) hist_sample<DIM>(D, hs, bins, K.hsum);
            if (A.abs_f && valid) A.abs_f[(int64_t)D.id * A.n_per_inst + idx] = isfinite(K.hsum) ? K.hsum : 0.0f;
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
// every compilation unit (Body::run loops over the samples inside each unit;
// with a leaf cache, Body::run first computes the cached leaf families of the
// P samples into shared memory, where every unit reads them):
// the unit's code is fetched once and then re-executed from the instruction
// cache for the other P - 1 samples, at no cost in registers.  The per-sample
// inputs live in local memory (SVS = 1) or, with SVS = T, in dynamic shared
// memory as [sample][thread] rows of FdSVT (sample p of this thread at
// V[p * SVS]); the tile histogram, when the launch provides it, follows them.
template <class Body, int N, int DIM, int R, int T, int P, int SVS = 1, int LCW = 0, bool LCG = false>
__device__ __forceinline__ void jit_main_loop(const EvalArgs &A) {
    __shared__ double acc[T / 32][R * 8];
    __shared__ int next_item;
    extern __shared__ float dyn_smem[];
    using FdSV = FdSVT<float, N>;
    constexpr int SV_FLOATS = SVS > 1 ? T * P * fd_sv_words(N) : 0;
    // leaf cache: LCW floats per sample, [float][sample p][thread], this thread's
    // column; in shared memory after the inputs, or (LCG) in this CTA's region
    // of a global scratch array (L2-resident)
    float *const LC = LCW == 0 ? nullptr
                    : LCG ? A.lc_global + (int64_t)blockIdx.x * (T * P * LCW) + threadIdx.x
                          : dyn_smem + SV_FLOATS + threadIdx.x;
    float *const hist_smem = dyn_smem + SV_FLOATS + (LCG ? 0 : T * P * LCW);
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
        const FdPar Q = fd_par(D);
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
            Body::run(V, Q, LC, cs, sn, K);
            if (A.abs_f) {
#pragma unroll
                for (int p = 0; p < P; ++p) {
                    const int64_t i = base + (int64_t)p * T + tid;
                    if (K[p].valid) A.abs_f[(int64_t)D.id * A.n_per_inst + i] = isfinite(K[p].hsum) ? K[p].hsum : 0.0f;
                }
            }
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
