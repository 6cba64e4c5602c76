// Host driver for the spline flow's per-sample device code (fd_nsf_math.cuh):
// the same functions the sampling, density and gradient kernels call, run on
// the CPU over a batch, so that a CPU test can compare them with the FP64
// oracle.  Input (binary): int32 dim, n_layers, n; FP32 parameters; FP32 x
// [dim][n]; FP32 w [n].  Output (binary): FP64 loss, FP64 gradient
// [n_params], FP32 z [dim][n], FP32 log q [n].
#include "fd_nsf_math.cuh"

#include <cstdio>
#include <vector>

using namespace nsf;

namespace {

struct HostAcc {
    double *g;
    void operator()(int64_t k, float v) { g[k] += v; }
};

// one layer's parameters in the staged layout (W1 and b1 rows padded to kPad)
std::vector<float> stage(const float *lp, int n_keep, int n_move) {
    std::vector<float> w(layer_smem_floats(n_keep, n_move), 0.0f);
    const int64_t head = head_floats(n_keep);
    for (int64_t k = 0; k < head; ++k) w[k] = lp[k];
    const int row = n_move * kParamsPerDim;
    for (int r = 0; r <= kHidden; ++r)
        for (int m = 0; m < n_move; ++m)
            for (int q = 0; q < kParamsPerDim; ++q)
                w[head + ((int64_t)r * n_move + m) * kPad + q] = lp[head + (int64_t)r * row + m * kParamsPerDim + q];
    return w;
}

bool read_all(FILE *f, void *p, size_t size, size_t count) { return fread(p, size, count, f) == count; }

}  // namespace

int main(int argc, char **argv) {
    if (argc != 3) return 2;
    FILE *f = fopen(argv[1], "rb");
    if (!f) return 3;
    int32_t hdr[3];
    if (!read_all(f, hdr, 4, 3)) return 4;
    const int D = hdr[0], L = hdr[1], n = hdr[2];
    if (D < 2 || D > kMaxDim || L < 1 || L > 16 || n < 1) return 5;
    const int64_t np = layer_offset(L, D);
    std::vector<float> P(np), X((size_t)n * D), W(n);
    if (!read_all(f, P.data(), 4, np) || !read_all(f, X.data(), 4, X.size()) || !read_all(f, W.data(), 4, n)) return 6;
    fclose(f);
    std::vector<std::vector<float>> staged(L);
    for (int l = 0; l < L; ++l) {
        const int n_keep = l % 2 == 0 ? D / 2 : D - D / 2;
        staged[l] = stage(P.data() + layer_offset(l, D), n_keep, D - n_keep);
    }
    double wsum = 0.0;
    for (float x : W) wsum += x;
    std::vector<double> G(np, 0.0);
    std::vector<float> Z((size_t)n * D), LQ(n);
    double loss = 0.0;
    for (int i = 0; i < n; ++i) {
        const float c = (float)(-(double)W[i] / wsum);
        float v[kMaxDim], vin[16][kMaxDim], vbar[kMaxDim];
        for (int j = 0; j < kMaxDim; ++j) {
            v[j] = j < D ? X[(size_t)j * n + i] : 0.5f;
            vbar[j] = 0.0f;
        }
        float logq = 0.0f;
        for (int l = L - 1; l >= 0; --l) {
            for (int j = 0; j < kMaxDim; ++j) vin[l][j] = v[j];
            logq -= layer_inverse(layer_at(staged[l].data(), l, D), v);
        }
        for (int j = 0; j < D; ++j) Z[(size_t)j * n + i] = v[j];
        LQ[i] = logq;
        loss += (double)c * logq;
        for (int l = 0; l < L; ++l) {
            HostAcc acc{G.data() + layer_offset(l, D)};
            layer_backward(layer_at(staged[l].data(), l, D), vin[l], vbar, c, acc);
        }
    }
    f = fopen(argv[2], "wb");
    if (!f) return 7;
    fwrite(&loss, 8, 1, f);
    fwrite(G.data(), 8, np, f);
    fwrite(Z.data(), 4, Z.size(), f);
    fwrite(LQ.data(), 4, n, f);
    fclose(f);
    return 0;
}
