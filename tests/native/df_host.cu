// Host driver for the double-float building blocks of fd_jit_rt.cuh that the
// order-1 G family uses: exp of a double-float argument (fd_exp_df) and the
// reciprocal of a double-float in [1, 2] (fd_df_rcp), so that a CPU test can
// compare them with high-precision references.
// Input (binary): int32 n; FP32 pairs (hi, lo) [n] for exp; FP32 pairs [n]
// for the reciprocal.  Output (binary): FP32 pairs [n] exp, then [n] rcp.
#include "fd_jit_rt.cuh"

#include <cstdio>
#include <vector>

int main(int argc, char **argv) {
    if (argc != 3) return 2;
    FILE *f = fopen(argv[1], "rb");
    if (!f) return 3;
    int32_t n = 0;
    if (fread(&n, 4, 1, f) != 1 || n < 0) return 4;
    std::vector<float> y(2 * (size_t)n), d(2 * (size_t)n), out(4 * (size_t)n);
    if (fread(y.data(), 4, y.size(), f) != y.size() || fread(d.data(), 4, d.size(), f) != d.size()) return 5;
    fclose(f);
    for (int32_t i = 0; i < n; ++i) {
        const FdDF e = fd_exp_df(FdDF{y[2 * i], y[2 * i + 1]});
        const FdDF r = fd_df_rcp(FdDF{d[2 * i], d[2 * i + 1]});
        out[2 * i] = e.hi;
        out[2 * i + 1] = e.lo;
        out[2 * (size_t)n + 2 * i] = r.hi;
        out[2 * (size_t)n + 2 * i + 1] = r.lo;
    }
    FILE *g = fopen(argv[2], "wb");
    if (!g) return 6;
    fwrite(out.data(), 4, out.size(), g);
    fclose(g);
    return 0;
}
