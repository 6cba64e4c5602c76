// Host driver for the integrand's per-sample device arithmetic
// (fd_jit_rt.cuh): the double-float sampler map and loop momenta, the leaf
// families (g_family, g_family_df, v_family) with the grid / remainder
// momentum sums and the time differences, the tape's FMA bundles, root
// accumulation and weighting, run on the CPU sample by sample as the tape
// interpreter does, so that a CPU test can compare them with the FP64 oracle.
// (The host build evaluates exp with the C library where the kernels use
// the MUFU approximation; everything else is the same FP32/FP64 code.)
//
// Input (binary): int32 n, dim, order, n_instr, n_slots, n_roots, nb (0: no
// VEGAS map); FP64 k_ext, mu, beta, Lambda, k_cut; u64 tape words [n_instr];
// u32 root words [n_roots] (n | m << 8 | l << 16 | dk << 24); FP32 hypercube
// points [dim][n]; with nb > 0 FP32 edges [dim][nb + 1].
// Output (binary): FP32 per-sample roots [n_roots][2][n] (Re, Im, weighted).
#include "fd_jit_rt.cuh"

#include <cmath>
#include <cstdio>
#include <vector>

namespace {

bool read_all(FILE *f, void *p, size_t size, size_t count) { return fread(p, size, count, f) == count; }

struct Par {
    float kext, kext_l, mu, mu_l, beta, beta_l, kc, kc_l, Lam, grid;
};

// the instance split of the library's host code (fd_integrand.cu)
Par split(double kext, double mu, double beta, double Lam, double kc) {
    Par P;
    int e = 0;
    (void)std::frexp(std::max(kc, kext), &e);
    const double g = std::ldexp(1.0, e - 13), g2 = g * g;
    const double kh = std::rint(kext / g) * g;
    const double mh = (double)(float)(std::rint(mu / g2) * g2);
    P.grid = (float)g;
    P.kext = (float)kh;
    P.kext_l = (float)(kext - kh);
    P.mu = (float)mh;
    P.mu_l = (float)(mu - mh);
    P.beta = (float)beta;
    P.beta_l = (float)(beta - (double)P.beta);
    P.kc = (float)kc;
    P.kc_l = (float)(kc - (double)P.kc);
    P.Lam = (float)Lam;
    return P;
}

constexpr int NK = FD_MAX_ORDER;

}  // namespace

int main(int argc, char **argv) {
    if (argc != 3) return 2;
    FILE *f = fopen(argv[1], "rb");
    if (!f) return 3;
    int32_t hdr[7];
    double prm[5];
    if (!read_all(f, hdr, 4, 7) || !read_all(f, prm, 8, 5)) return 4;
    const int n = hdr[0], dim = hdr[1], N = hdr[2], n_instr = hdr[3], n_slots = hdr[4], R = hdr[5], nb = hdr[6];
    std::vector<uint64_t> tape(n_instr);
    std::vector<uint32_t> roots(R);
    std::vector<float> x((size_t)dim * n), edges(nb ? (size_t)dim * (nb + 1) : 0);
    if (!read_all(f, tape.data(), 8, tape.size()) || !read_all(f, roots.data(), 4, roots.size()) ||
        !read_all(f, x.data(), 4, x.size()) || (nb && !read_all(f, edges.data(), 4, edges.size())))
        return 5;
    fclose(f);
    const Par P = split(prm[0], prm[1], prm[2], prm[3], prm[4]);
    FdTab4 tab[257];
    for (int q = 0; q <= 256; ++q) {
        const double a = 2.0 * M_PI * (double)q / 256.0;
        const double c = std::cos(a), s = std::sin(a);
        tab[q].x = (float)c;
        tab[q].y = (float)(c - (double)tab[q].x);
        tab[q].z = (float)s;
        tab[q].w = (float)(s - (double)tab[q].z);
    }
    std::vector<float> out((size_t)R * 2 * n, 0.0f);
    std::vector<float> S(n_slots + 2);
    for (int i = 0; i < n; ++i) {
        // ---- sample point (sample_point / prologue) ----
        FdDF xd[FD_MAX_DIM];
        float jd[FD_MAX_DIM];
        for (int d = 0; d < dim; ++d) {
            xd[d] = FdDF{x[(size_t)d * n + i], 0.0f};
            jd[d] = 1.0f;
            if (nb) (void)fd_vegas_df(xd[d].hi, nb, edges.data() + (size_t)d * (nb + 1), xd[d], jd[d]);
        }
        float kx[NK] = {}, ky[NK] = {}, kz[NK] = {}, kxl[NK] = {}, kyl[NK] = {}, kzl[NK] = {};
        float t[NK] = {}, tl[NK] = {}, jac[NK] = {};
        float w = 1.0f;
        for (int j = 0; j < N; ++j) {
            const int c0 = (j == 0) ? 0 : 4 * j - 1;
            float kh[3], kl[3];
            const float r = fd_loop_momentum(xd[c0], xd[c0 + 1], xd[c0 + 2], FdDF{P.kc, P.kc_l}, tab, P.grid,
                                             1.0f / P.grid, kh, kl);
            kx[j] = kh[0];
            ky[j] = kh[1];
            kz[j] = kh[2];
            kxl[j] = kl[0];
            kyl[j] = kl[1];
            kzl[j] = kl[2];
            w *= P.kc * r * r * FD_INV_2PI2;
            w *= jd[c0] * jd[c0 + 1] * jd[c0 + 2];
            if (j >= 1) {
                t[j] = xd[4 * j + 2].hi;
                tl[j] = xd[4 * j + 2].lo;
                w *= P.beta * jd[4 * j + 2];
            }
            jac[j] = w;
        }
        // ---- the tape (interpreter order) ----
        S[0] = 0.0f;
        S[1] = 1.0f;
        for (int j = 0; j < N; ++j) S[2 + j] = t[j];
        float re = 0.0f, im = 0.0f;
        for (int k = 0; k < n_instr; ++k) {
            const uint64_t wd = tape[k];
            const uint32_t op = (uint32_t)(wd & 63u);
            if (op == 8u) {   // bundle: all operands first
                const int nbd = (int)((wd >> 6) & 15u);
                float v[8];
                int dst[8];
                for (int q = 0; q < nbd; ++q) {
                    const uint64_t m = tape[k + 1 + q];
                    dst[q] = (int)(m & 0xFFFFu);
                    v[q] = fmaf(S[(m >> 16) & 0xFFFFu], S[(m >> 32) & 0xFFFFu], S[(m >> 48) & 0xFFFFu]);
                }
                for (int q = 0; q < nbd; ++q) S[dst[q]] = v[q];
                k += nbd;
                continue;
            }
            if (op == 63u) break;
            const uint32_t d = (uint32_t)(wd >> 6) & 16383u, a = (uint32_t)(wd >> 20) & 16383u;
            if (op == 2u || op == 3u) {
                const uint32_t la = (uint32_t)(wd >> 34) & 7u, lb = (uint32_t)(wd >> 37) & 7u;
                const int M = (int)((wd >> 40) & 7u), dk = (int)((wd >> 43) & 1u);
                float cf[NK + 1];
                for (int j = 0; j <= NK; ++j) cf[j] = (float)(((int)(a << (30 - 2 * j))) >> 30);
                const float ks = cf[0];
                float h[3] = {0.0f, 0.0f, cf[0] * P.kext}, l[3] = {0.0f, 0.0f, cf[0] * P.kext_l};
                for (int j = 0; j < NK; ++j) {
                    h[0] = fmaf(cf[j + 1], kx[j], h[0]);
                    h[1] = fmaf(cf[j + 1], ky[j], h[1]);
                    h[2] = fmaf(cf[j + 1], kz[j], h[2]);
                    l[0] = fmaf(cf[j + 1], kxl[j], l[0]);
                    l[1] = fmaf(cf[j + 1], kyl[j], l[1]);
                    l[2] = fmaf(cf[j + 1], kzl[j], l[2]);
                }
                auto put = [&](int j, float v) { S[d + j] = v; };
                if (op == 2u) {
                    float dxh, dxl;
                    fd_time_diff(t[la], tl[la], t[lb], tl[lb], dxh, dxl);
                    if ((wd >> FD_LEAF_PRECISE_BIT) & 1u) {
                        g_family_df(h[0], h[1], h[2], FdDF{l[0], 0.0f}, FdDF{l[1], 0.0f}, FdDF{l[2], 0.0f}, ks,
                                    dxh, dxl, P.beta, P.beta_l, P.mu, P.mu_l, M, dk, put);
                    } else {
                        const float eps = fd_eps(h[0], h[1], h[2], l[0], l[1], l[2], P.mu, P.mu_l);
                        g_family<float>(eps, h[2] + l[2], ks, dxh, dxl, P.beta, M, dk, put);
                    }
                } else {
                    const float qx = h[0] + l[0], qy = h[1] + l[1], qz = h[2] + l[2];
                    const float q2 = fmaf(qx, qx, fmaf(qy, qy, qz * qz));
                    v_family<float>(q2, qz, ks, P.Lam, M, dk, put);
                }
            } else if (op == 4u) {   // root accumulate
                const uint32_t line = (uint32_t)(wd >> 34) & 7u;
                float cs = 1.0f, sn = 0.0f;
                if (line) {
                    cs = (float)std::cos(M_PI * (double)t[line]);
                    sn = (float)std::sin(M_PI * (double)t[line]);
                }
                re = fmaf(S[a], cs, re);
                im = fmaf(S[a], sn, im);
            } else if (op == 5u) {   // root complete
                const int r = (int)d;
                const float J = jac[(roots[r] & 255u) - 1];
                out[((size_t)r * 2) * n + i] = re * J;
                out[((size_t)r * 2 + 1) * n + i] = im * J;
                re = im = 0.0f;
            } else if (op == 6u) {
                const uint32_t bits = (uint32_t)(wd >> 32);
                float v;
                memcpy(&v, &bits, 4);
                S[d] = v;
            }
        }
    }
    FILE *o = fopen(argv[2], "wb");
    if (!o) return 6;
    fwrite(out.data(), 4, out.size(), o);
    fclose(o);
    return 0;
}
