// Host driver for the sampler map's double-float kinematics (fd_jit_rt.cuh):
// the loop momenta of a batch of hypercube points, as the kernels compute them
// (grid part + remainder of each component, summed here in FP64), so that a
// CPU test can compare them with the oracle's FP64 map.
// Input (binary): int32 n, order; FP64 K_c; FP32 points [4 order - 1][n].
// Output (binary): FP64 momenta [order][3][n].
#include "fd_jit_rt.cuh"

#include <cmath>
#include <cstdio>
#include <vector>

int main(int argc, char **argv) {
    if (argc != 3) return 2;
    FILE *f = fopen(argv[1], "rb");
    if (!f) return 3;
    int32_t hdr[2];
    double kc = 0.0;
    if (fread(hdr, 4, 2, f) != 2 || fread(&kc, 8, 1, f) != 1) return 4;
    const int n = hdr[0], N = hdr[1], dim = 4 * N - 1;
    std::vector<float> x((size_t)dim * n);
    if (fread(x.data(), 4, x.size(), f) != x.size()) return 5;
    fclose(f);
    FdTab4 tab[257];
    for (int q = 0; q <= 256; ++q) {
        const double a = 2.0 * M_PI * (double)q / 256.0;
        tab[q].x = (float)std::cos(a);
        tab[q].y = (float)(std::cos(a) - (double)tab[q].x);
        tab[q].z = (float)std::sin(a);
        tab[q].w = (float)(std::sin(a) - (double)tab[q].z);
    }
    int e = 0;
    (void)std::frexp(kc, &e);
    const float g = (float)std::ldexp(1.0, e - 13);
    const FdDF kcd{(float)kc, (float)(kc - (double)(float)kc)};
    std::vector<double> out((size_t)N * 3 * n);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < N; ++j) {
            const int c0 = (j == 0) ? 0 : 4 * j - 1;
            const FdDF a{x[(size_t)c0 * n + i], 0.0f}, b{x[(size_t)(c0 + 1) * n + i], 0.0f},
                c{x[(size_t)(c0 + 2) * n + i], 0.0f};
            float kh[3], kl[3];
            (void)fd_loop_momentum(a, b, c, kcd, tab, g, 1.0f / g, kh, kl);
            for (int q = 0; q < 3; ++q) out[((size_t)j * 3 + q) * n + i] = (double)kh[q] + (double)kl[q];
        }
    FILE *o = fopen(argv[2], "wb");
    if (!o) return 6;
    fwrite(out.data(), 8, out.size(), o);
    fclose(o);
    return 0;
}
