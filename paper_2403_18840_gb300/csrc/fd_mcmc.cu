// NF-MCMC / VEGAS-MCMC chains (Sec. V, Eqs. target_distr and
// nf_mcmc_estimator): independence Metropolis-Hastings over proposals x ~ q
// that the integrand kernels have already evaluated.
//
// Target pi = alpha q + (1 - alpha) |f|, proposals from q independently of the
// chain's state, acceptance R = min{1, pi(x') q(x_t) / (pi(x_t) q(x'))},
// estimator I = sum f/pi / sum q/pi over the visited states.  Through the
// importance weight w = f/q of a proposal, g = pi/q = alpha + (1 - alpha)|w|_p,
// R = g'/g_t, f/pi = w/g and q/pi = 1/g, so a step needs the proposal's
// weights only.  Because the proposals do not depend on the chain, all of them
// are generated and evaluated in bulk by the sampler and integrand kernels
// (full-GPU batches); the chains then run here as one thread each over their
// columns of the weight matrix, a memory-bound pass (coalesced: proposal k of
// chain c is column k * n_chains + c).
//
// The step's arithmetic is FP64 with every operation explicitly rounded
// (no multiply-add contraction), in the order the definitions give, so the
// chains are reproducible bit for bit by any implementation that rounds each
// operation the same way.
#include "fd_internal.cuh"

namespace {

constexpr int kMaxOut = 32;                  // weight components per proposal
constexpr uint32_t kChainTag = 0x40000000u;  // acceptance-uniform stream: counter word 3 = tag | (step >> 2)

// NO >= n_out: the size of the per-chain register arrays
template <int NO>
__global__ void __launch_bounds__(128) mcmc_chain_kernel(const float *__restrict__ w, int n_out, int64_t ld,
                                                         int n_sel, int64_t n_chains, int n_steps, double alpha,
                                                         uint32_t seed_lo, uint32_t seed_hi, uint32_t iter,
                                                         int n_therm, double *state, double *sums) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n_chains) return;
    // cur: the state's weights; m_q = 1/g (q/pi) and m_w = cur m_q (f/pi) of
    // the state, computed when it is accepted (the same operands and rounding
    // as at every later step, so measuring them from the cache changes no bit)
    double cur[NO], acc_w[NO], m_w[NO];
    double g = state[(int64_t)n_out * n_chains + c];
    double m_q = g != 0.0 ? __ddiv_rn(1.0, g) : 0.0;
#pragma unroll
    for (int o = 0; o < NO; ++o) {
        cur[o] = o < n_out ? state[(int64_t)o * n_chains + c] : 0.0;
        m_w[o] = __dmul_rn(cur[o], m_q);
        acc_w[o] = 0.0;
    }
    double acc_q = 0.0, n_acc = 0.0;
    const double one_m_alpha = __dadd_rn(1.0, -alpha);
    u32x4 words{0u, 0u, 0u, 0u};
    // The proposals' weights do not depend on the chain: load those of the
    // next B steps before stepping through them (a chain's steps are
    // sequential, so this hides the loads' latency behind the FP64 work)
    constexpr int B = NO <= 2 ? 8 : NO <= 4 ? 4 : NO <= 8 ? 2 : 1;
    for (int k0 = 0; k0 < n_steps; k0 += B) {
        float wb[B][NO];
#pragma unroll
        for (int j = 0; j < B; ++j)
#pragma unroll
            for (int o = 0; o < NO; ++o)
                wb[j][o] = (k0 + j < n_steps && o < n_out)
                               ? __ldg(w + (int64_t)(k0 + j) * n_chains + c + (int64_t)o * ld)
                               : 0.0f;
#pragma unroll
        for (int j = 0; j < B; ++j) {
            const int k = k0 + j;
            if (k >= n_steps) break;
            if ((k & 3) == 0)
                words = philox4x32_10(
                    u32x4{(uint32_t)c, (uint32_t)((uint64_t)c >> 32), iter, kChainTag | (uint32_t)(k >> 2)}, seed_lo,
                    seed_hi);
            const uint32_t word = (k & 3) == 0 ? words.x : (k & 3) == 1 ? words.y : (k & 3) == 2 ? words.z : words.w;
            const double u = (double)word_to_uniform(word);
            double s = 0.0;
#pragma unroll
            for (int o = 0; o < NO; ++o)
                if (o < n_sel) s = __dadd_rn(s, fabs((double)wb[j][o]));
            const double gp = __dadd_rn(alpha, __dmul_rn(one_m_alpha, s));      // pi/q of the proposal
            // u < R = g'/g_t, as u g_t < g' (g_t > 0 once the chain has a state)
            const bool accept = g == 0.0 || __dmul_rn(u, g) < gp;
            if (accept) {
                g = gp;
                m_q = __ddiv_rn(1.0, g);
#pragma unroll
                for (int o = 0; o < NO; ++o)
                    if (o < n_out) {
                        cur[o] = (double)wb[j][o];
                        m_w[o] = __dmul_rn(cur[o], m_q);
                    }
                n_acc += 1.0;
            }
            if (k >= n_therm) {
#pragma unroll
                for (int o = 0; o < NO; ++o)
                    if (o < n_out) acc_w[o] = __dadd_rn(acc_w[o], m_w[o]);   // f/pi
                acc_q = __dadd_rn(acc_q, m_q);                              // q/pi
            }
        }
    }
#pragma unroll
    for (int o = 0; o < NO; ++o)
        if (o < n_out) {
            state[(int64_t)o * n_chains + c] = cur[o];
            sums[(int64_t)o * n_chains + c] = acc_w[o];
        }
    state[(int64_t)n_out * n_chains + c] = g;
    sums[(int64_t)n_out * n_chains + c] = acc_q;
    sums[(int64_t)(n_out + 1) * n_chains + c] = n_acc;
}

// Fixed-order block sum of one value per thread (256 threads).
__device__ double block_sum(double v, double *red) {
    red[threadIdx.x] = v;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) red[threadIdx.x] = __dadd_rn(red[threadIdx.x], red[threadIdx.x + h]);
        __syncthreads();
    }
    const double r = red[0];
    __syncthreads();
    return r;
}

// One block per component o: I_o = sum_c A_oc / sum_c B_c and the delta-method
// variance sum_c (A_oc - I_o B_c)^2 / (C (C - 1)) / mean(B)^2; block n_out: the
// acceptance fraction.  Every thread walks a fixed stride of chains, then a
// fixed tree: the result does not depend on scheduling.
__global__ void __launch_bounds__(256) mcmc_estimate_kernel(const double *__restrict__ sums, int n_out,
                                                            int64_t n_chains, int n_steps, double *out) {
    __shared__ double red[256];
    const int o = blockIdx.x;
    const double *B = sums + (int64_t)n_out * n_chains;
    if (o == n_out) {
        double a = 0.0;
        for (int64_t c = threadIdx.x; c < n_chains; c += 256) a += sums[(int64_t)(n_out + 1) * n_chains + c];
        a = block_sum(a, red);
        if (threadIdx.x == 0) {
            out[2 * n_out] = a / ((double)n_chains * (double)n_steps);
            out[2 * n_out + 1] = 0.0;
        }
        return;
    }
    const double *A = sums + (int64_t)o * n_chains;
    double sa = 0.0, sb = 0.0;
    for (int64_t c = threadIdx.x; c < n_chains; c += 256) {
        sa += A[c];
        sb += B[c];
    }
    sa = block_sum(sa, red);
    sb = block_sum(sb, red);
    const double I = sa / sb;
    double sr = 0.0;
    for (int64_t c = threadIdx.x; c < n_chains; c += 256) {
        const double r = A[c] - I * B[c];
        sr += r * r;
    }
    sr = block_sum(sr, red);
    if (threadIdx.x == 0) {
        const double C = (double)n_chains, mean_b = sb / C;
        out[2 * o] = I;
        out[2 * o + 1] = sr / (C * (C - 1.0)) / (mean_b * mean_b);
    }
}

}  // namespace

extern "C" fd_status fd_mcmc_chains(const float *w, int32_t n_out, int64_t ld, int32_t n_sel, int64_t n_chains,
                                    int32_t n_steps, double alpha, uint64_t seed, uint64_t iter, int32_t n_therm,
                                    double *state, double *sums, void *stream) {
    FD_REQUIRE(w && state && sums, "w, state and sums are required");
    FD_REQUIRE(n_out >= 1 && n_out <= kMaxOut, "n_out must be in [1, 32]");
    FD_REQUIRE(n_sel >= 1 && n_sel <= n_out, "n_sel must be in [1, n_out]");
    FD_REQUIRE(n_chains >= 1 && n_chains <= (int64_t(1) << 31), "n_chains must be in [1, 2^31]");
    FD_REQUIRE(n_steps >= 1 && n_therm >= 0, "n_steps must be positive and n_therm non-negative");
    FD_REQUIRE(ld >= n_chains * (int64_t)n_steps, "ld must hold n_chains * n_steps proposals");
    FD_REQUIRE(alpha > 0.0 && alpha <= 1.0, "alpha must be in (0, 1]");
    // chains are sequential and FP64-bound: spread them over every SM (down to
    // one warp per block) before stacking warps on one SM's FP64 pipe
    int dev = 0, n_sm = 1;
    FD_CHECK_CUDA(cudaGetDevice(&dev));
    FD_CHECK_CUDA(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
    const int64_t per_sm = (n_chains + n_sm - 1) / n_sm;
    const int threads = per_sm <= 32 ? 32 : per_sm <= 64 ? 64 : 128;
    const unsigned blocks = (unsigned)((n_chains + threads - 1) / threads);
    const cudaStream_t st = (cudaStream_t)stream;
    const uint32_t lo = (uint32_t)seed, hi = (uint32_t)(seed >> 32), it = (uint32_t)iter;
#define FD_MCMC_LAUNCH(NO)                                                                                      \
    mcmc_chain_kernel<NO><<<blocks, threads, 0, st>>>(w, n_out, ld, n_sel, n_chains, n_steps, alpha, lo, hi, it, \
                                                  n_therm, state, sums)
    if (n_out <= 2)
        FD_MCMC_LAUNCH(2);
    else if (n_out <= 4)
        FD_MCMC_LAUNCH(4);
    else if (n_out <= 8)
        FD_MCMC_LAUNCH(8);
    else if (n_out <= 16)
        FD_MCMC_LAUNCH(16);
    else
        FD_MCMC_LAUNCH(32);
#undef FD_MCMC_LAUNCH
    FD_CHECK_CUDA(cudaGetLastError());
    return FD_OK;
}

extern "C" fd_status fd_mcmc_estimate(const double *sums, int32_t n_out, int64_t n_chains, int32_t n_steps,
                                      double *out, void *stream) {
    FD_REQUIRE(sums && out, "sums and out are required");
    FD_REQUIRE(n_out >= 1 && n_out <= kMaxOut, "n_out must be in [1, 32]");
    FD_REQUIRE(n_chains >= 2 && n_steps >= 1, "at least two chains and one step");
    mcmc_estimate_kernel<<<n_out + 1, 256, 0, (cudaStream_t)stream>>>(sums, n_out, n_chains, n_steps, out);
    FD_CHECK_CUDA(cudaGetLastError());
    return FD_OK;
}
