// Batched integrand evaluation: Philox -> sampler map -> (k, tau) -> leaf
// families -> tape contraction -> weighted roots -> FP64 tile partials.
//
// What one sample computes is fixed by the paper's Eq. sigma_integration
// (order-n self-energy as an n(d+1)-dimensional integral summed over
// topologies) with the counterterm expansion of Eq. sigma_xi_dmu_dlambda:
// every root of the compiled graph is a Taylor coefficient
// d^m_mu d^l_Lambda (d_k)^dk of the diagram sum, evaluated at the sample
// point and multiplied by the Jacobian of the hypercube map and by
// exp(i w0 tau_out) with w0 = pi / beta.
//
// Execution model (sm_103a):
//  * persistent CTAs walk work items = (instance, tile of FD_TILE_SAMPLES
//    consecutive samples); each thread owns one sample per pass;
//  * per-sample state lives in shared memory as [slot][thread] FP32 words
//    (a warp touches 32 consecutive words per slot: conflict-free);
//  * the graph tape (64-bit instructions, identical for all samples) is
//    streamed into a double buffer of shared memory by 1-D TMA bulk copies
//    completing on mbarriers (bounded waits), then broadcast-read by all
//    threads;
//  * roots are reduced per pass with warp shuffles (FP32) and accumulated per
//    warp in FP64 with Neumaier compensation; at the end of a work item the
//    warps are combined in a fixed order into the tile's partial sums.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <string>
#include <vector>

#include "fd_internal.cuh"

namespace {

constexpr int CHUNK_INSTR = 2048;                     // 16 KB per tape buffer
constexpr int CHUNK_BYTES = CHUNK_INSTR * 8;
constexpr uint32_t WAIT_LIMIT = 1u << 24;             // polls before a tape wait gives up
constexpr float K_INV_2PI2 = 0.050660591821168885f;    // 1 / (2 pi^2)
constexpr float K_8PI = 25.132741228718345f;

struct InstDesc {
    const uint64_t *tape;      // instruction words (device)
    const uint32_t *roots;     // root table (device)
    const float *edges;        // VEGAS FP32 edges [dim][nb+1] or null
    double *hist;              // VEGAS histogram [dim][nb] or null
    const float *points;       // explicit points [dim_max][n] or null
    const float *point_w;      // explicit weights [n] or null
    int32_t n_instr, n_slots, order, dim, n_roots, n_bins;
    float kext, mu, beta, Lambda, kc;
    float pad;
};

struct EvalArgs {
    int32_t n_inst, tiles_per_inst, r_max, slots_total, dim_max;
    int64_t n_per_inst;
    uint32_t seed_lo, seed_hi, iter;
    double *partials;
    float *per_sample_f;
    int *status;
    InstDesc inst[FD_MAX_INST];
};

struct SmemLayout {
    // byte offsets inside dynamic shared memory
    int tape0, tape1, bars, acc, slots, total;
};

__host__ __device__ inline SmemLayout smem_layout(int threads, int slots_total, int r_max) {
    SmemLayout L;
    L.tape0 = 0;
    L.tape1 = CHUNK_BYTES;
    L.bars = 2 * CHUNK_BYTES;
    L.acc = L.bars + 16;                                     // 8-byte aligned
    const int nwarps = threads / 32;
    L.slots = L.acc + nwarps * r_max * 4 * 2 * 8;            // (sum, sumsq) x (re, im) x (value, comp)
    L.slots = (L.slots + 15) & ~15;
    L.total = L.slots + slots_total * threads * 4;
    return L;
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

template <int T>
struct Slots {
    float *base;   // &slots[tid]
    __device__ __forceinline__ float &operator[](uint32_t s) const { return base[s * T]; }
};

// G0 Taylor family: c_j = (d/dmu)^j G0 / j!, j <= M (+ d/dk copies).
// Written as sign * exp(-eps tau*) * phi(eps - dmu) with the Fermi factor
// phi >= 1/2 (phi = 1 - f for eps >= 0, f for eps < 0) and tau* the matching
// antiperiodic time, so the exponent is never positive.  The series of
// phi(eps - d) follows from the logistic ODE d phi / d eps = +-beta phi (1 - phi)
// (Taylor-mode recurrence); the series of exp(d tau*) is tau*^k / k!.
template <int T>
__device__ __forceinline__ void g_leaf(const Slots<T> &S, uint64_t w, float beta) {
    const uint32_t d = ins_d(w), a = ins_a(w), b = ins_b(w), c = ins_c(w), imm = ins_imm(w);
    const int M = (int)(imm & 7u);
    const int dk = (int)((imm >> 3) & 1u);
    const float ks = (float)((int)((imm >> 4) & 3u) - 1);
    const float eps = S[a], phi = S[a + 1], psi = S[a + 2], pz = S[a + 3];
    const float dx = S[b] - S[c];
    const bool pos = dx > 0.0f;
    const float tau = beta * dx;
    const bool occ = eps < 0.0f;
    const float tstar = occ ? (pos ? tau - beta : tau) : (pos ? tau : tau + beta);
    const float sgn = pos ? -1.0f : 1.0f;
    const float X = sgn * __expf(-eps * tstar) * phi;
    if (M == 0 && !dk) {
        S[d] = X;
        return;
    }
    const int Mx = M + dk;
    // Phi_hat (series of phi(eps - d) / phi) and A (series of exp(d tau*))
    float ph[FD_MAX_M + 1], ps[FD_MAX_M + 1], A[FD_MAX_M + 1], cf[FD_MAX_M + 1];
    const float g = occ ? beta : -beta;
    ph[0] = 1.0f;
    ps[0] = psi;
    A[0] = 1.0f;
#pragma unroll
    for (int k = 0; k < FD_MAX_M; ++k) {
        if (k < Mx) {
            float s = 0.0f;
#pragma unroll
            for (int i = 0; i <= k; ++i) s = fmaf(ph[i], ps[k - i], s);
            ph[k + 1] = g * s / (float)(k + 1);
            ps[k + 1] = -phi * ph[k + 1];
            A[k + 1] = A[k] * tstar / (float)(k + 1);
        }
    }
#pragma unroll
    for (int j = 0; j <= FD_MAX_M; ++j) {
        if (j <= Mx) {
            float s = 0.0f;
#pragma unroll
            for (int i = 0; i <= j; ++i) s = fmaf(A[j - i], ph[i], s);
            cf[j] = X * s;
        }
    }
#pragma unroll
    for (int j = 0; j <= FD_MAX_M; ++j)
        if (j <= M) S[d + j] = cf[j];
    if (dk) {
        const float kz = -2.0f * ks * pz;
#pragma unroll
        for (int j = 0; j < FD_MAX_M; ++j)
            if (j <= M) S[d + M + 1 + j] = kz * (float)(j + 1) * cf[j + 1];
    }
}

// V Taylor family: c_l = (d/dLambda)^l V / l! = 8 pi (-1)^l w^(l+1), w = 1/(q^2+Lambda)
template <int T>
__device__ __forceinline__ void v_leaf(const Slots<T> &S, uint64_t w, float Lambda) {
    const uint32_t d = ins_d(w), a = ins_a(w), imm = ins_imm(w);
    const int L = (int)(imm & 7u);
    const int dk = (int)((imm >> 3) & 1u);
    const float ks = (float)((int)((imm >> 4) & 3u) - 1);
    const float q2 = S[a + 3], pz = S[a + 2];
    const float inv = __frcp_rn(q2 + Lambda);
    float cl = K_8PI * inv;
    float cf[FD_MAX_M + 1];
#pragma unroll
    for (int l = 0; l <= FD_MAX_M; ++l) {
        if (l <= L + dk) {
            cf[l] = cl;
            cl = -inv * cl;
        }
    }
#pragma unroll
    for (int l = 0; l <= FD_MAX_M; ++l)
        if (l <= L) S[d + l] = cf[l];
    if (dk) {
        const float kz = 2.0f * ks * pz;
#pragma unroll
        for (int l = 0; l < FD_MAX_M; ++l)
            if (l <= L) S[d + L + 1 + l] = kz * (float)(l + 1) * cf[l + 1];
    }
}

template <int T>
__device__ __forceinline__ bool run_chunk(const Slots<T> &S, const uint64_t *code, int cnt,
                                          const InstDesc &D) {
    for (int k = 0; k < cnt; ++k) {
        const uint64_t w = code[k];
        switch (ins_op(w)) {
            case OP_MUL:
                S[ins_d(w)] = S[ins_a(w)] * S[ins_b(w)];
                break;
            case OP_FMA:
                S[ins_d(w)] = fmaf(S[ins_a(w)], S[ins_b(w)], S[ins_c(w)]);
                break;
            case OP_ADD:
                S[ins_d(w)] = S[ins_a(w)] + S[ins_b(w)];
                break;
            case OP_MULC:
                S[ins_d(w)] = S[ins_a(w)] * __uint_as_float(ins_hi(w));
                break;
            case OP_CONST:
                S[ins_d(w)] = __uint_as_float(ins_hi(w));
                break;
            case OP_GLEAF:
                g_leaf(S, w, D.beta);
                break;
            case OP_VLEAF:
                v_leaf(S, w, D.Lambda);
                break;
            case OP_FERMI: {
                const uint32_t d = ins_d(w), a = ins_a(w);
                const float eps = S[a + 3] - D.mu;
                const float E = __expf(-D.beta * fabsf(eps));
                const float phi = __frcp_rn(1.0f + E);
                S[d] = eps;
                S[d + 1] = phi;
                S[d + 2] = E * phi;
                S[d + 3] = S[a + 2];
                break;
            }
            case OP_MOM: {
                const uint32_t d = ins_d(w), a = ins_a(w), b = ins_b(w);
                const float sg = (ins_imm(w) & 1u) ? -1.0f : 1.0f;
                const float px = fmaf(sg, S[b], S[a]);
                const float py = fmaf(sg, S[b + 1], S[a + 1]);
                const float pz = fmaf(sg, S[b + 2], S[a + 2]);
                S[d] = px;
                S[d + 1] = py;
                S[d + 2] = pz;
                S[d + 3] = fmaf(px, px, fmaf(py, py, pz * pz));
                break;
            }
            case OP_ROOT: {
                const uint32_t d = ins_d(w);
                const float v = S[ins_a(w)];
                S[d] = fmaf(v, S[ins_b(w)], S[d]);
                S[d + 1] = fmaf(v, S[ins_c(w)], S[d + 1]);
                break;
            }
            case OP_ROOT0:
                S[ins_d(w)] += S[ins_a(w)];
                break;
            case OP_END:
                return true;
            default:
                break;
        }
    }
    return false;
}

// Fixed part of the per-sample state (the tape's prologue slots) plus the
// extra slots [n_slots, n_slots + order) holding the Jacobian of each root
// order and [n_slots + order, + dim) holding the VEGAS bins.
template <int T>
__device__ __forceinline__ void prologue(const Slots<T> &S, const InstDesc &D, const EvalArgs &A,
                                         int64_t i, int inst) {
    const int N = D.order, dim = D.dim;
    float x[FD_MAX_DIM];
    float jv_prefix = 1.0f;    // VEGAS / point weight over the dims consumed so far
    float jn[FD_MAX_ORDER + 1];
    if (D.points) {
#pragma unroll
        for (int d = 0; d < FD_MAX_DIM; ++d)
            if (d < dim) x[d] = D.points[(int64_t)d * A.n_per_inst + i];
        jv_prefix = D.point_w ? D.point_w[i] : 1.0f;
    } else {
        const uint32_t c0 = (uint32_t)(uint64_t)i, c1 = (uint32_t)((uint64_t)i >> 32);
#pragma unroll
        for (int blk = 0; blk < (FD_MAX_DIM + 3) / 4; ++blk) {
            if (4 * blk < dim) {
                const u32x4 r = philox4x32_10(u32x4{c0, c1, A.iter, ((uint32_t)inst << 8) | (uint32_t)blk},
                                              A.seed_lo, A.seed_hi);
                const uint32_t wv[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (4 * blk + q < FD_MAX_DIM) x[4 * blk + q] = word_to_uniform(wv[q]);
            }
        }
    }
    // VEGAS map per dimension (bins kept for the histogram)
    float jd[FD_MAX_DIM];
#pragma unroll
    for (int d = 0; d < FD_MAX_DIM; ++d) {
        jd[d] = 1.0f;
        if (d < dim && D.edges) {
            const int nb = D.n_bins;
            const float y = x[d] * (float)nb;
            int bin = min((int)y, nb - 1);
            const float *e = D.edges + (int64_t)d * (nb + 1);
            const float lo = __ldg(e + bin), hi = __ldg(e + bin + 1);
            x[d] = fmaf(y - (float)bin, hi - lo, lo);
            jd[d] = (float)nb * (hi - lo);
            S[D.n_slots + N + d] = __int_as_float(bin);
        }
    }
    // k_ext record and constant zero
    S[0] = 0.0f;
    S[1] = 0.0f;
    S[2] = 0.0f;
    S[3] = D.kext;
    S[4] = D.kext * D.kext;
    const int t0 = 5 + 4 * N;
    const int p0 = t0 + N - 1;
    float jac = 1.0f;
    int used = 0;    // hypercube coordinates consumed
#pragma unroll
    for (int j = 1; j <= FD_MAX_ORDER; ++j) {
        if (j <= N) {
            const int c0 = (j == 1) ? 0 : 4 * j - 5;
            const float xa = x[c0], xb = x[c0 + 1], xc = x[c0 + 2];
            const float r = D.kc * xa;
            const float cth = fmaf(2.0f, xb, -1.0f);
            const float sth = 2.0f * sqrtf(xb * (1.0f - xb));
            float sp, cp;
            sincospif(2.0f * xc, &sp, &cp);
            const int rec = 5 + 4 * (j - 1);
            S[rec] = r * sth * cp;
            S[rec + 1] = r * sth * sp;
            S[rec + 2] = r * cth;
            S[rec + 3] = r * r;
            jac *= D.kc * r * r * K_INV_2PI2;
            jv_prefix *= D.points ? 1.0f : jd[c0] * jd[c0 + 1] * jd[c0 + 2];
            used = c0 + 3;
            if (j >= 2) {
                const float xt = x[4 * j - 2];
                S[t0 + j - 2] = xt;
                float st, ct;
                sincospif(xt, &st, &ct);
                S[p0 + 2 * (j - 2)] = ct;
                S[p0 + 2 * (j - 2) + 1] = st;
                jac *= D.beta;
                jv_prefix *= D.points ? 1.0f : jd[4 * j - 2];
                used = 4 * j - 1;
            }
            S[D.n_slots + j - 1] = jac * jv_prefix;
        }
    }
    (void)used;
    (void)jn;
}

template <int T>
__global__ void __launch_bounds__(T) integrand_kernel(const __grid_constant__ EvalArgs A) {
    extern __shared__ __align__(16) unsigned char smem[];
    const SmemLayout L = smem_layout(T, A.slots_total, A.r_max);
    uint64_t *buf[2] = {reinterpret_cast<uint64_t *>(smem + L.tape0),
                        reinterpret_cast<uint64_t *>(smem + L.tape1)};
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + L.bars);
    double *acc = reinterpret_cast<double *>(smem + L.acc);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const Slots<T> S{reinterpret_cast<float *>(smem + L.slots) + tid};
    const int n_items = A.n_inst * A.tiles_per_inst;
    const int racc = A.r_max * 4;   // doubles per warp for values (sum, sumsq) x (re, im)

    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_mbarrier_init();
    }
    __syncthreads();
    uint32_t phase[2] = {0u, 0u};   // completed loads per buffer (parity source)
    bool failed = false;

    for (int item = blockIdx.x; item < n_items && !failed; item += gridDim.x) {
        const int inst = item / A.tiles_per_inst;
        const int tile = item % A.tiles_per_inst;
        const InstDesc &D = A.inst[inst];
        const int n_chunks = (D.n_instr + CHUNK_INSTR - 1) / CHUNK_INSTR;
        // zero the per-warp accumulators
        for (int k = tid; k < (T / 32) * racc * 2; k += T) acc[k] = 0.0;
        const int64_t first = (int64_t)tile * FD_TILE_SAMPLES;
        const int64_t last = min(first + (int64_t)FD_TILE_SAMPLES, A.n_per_inst);
        const int passes = (int)((last - first + T - 1) / T);
        // start streaming: chunk g of the cyclic sequence (pass-major) goes to buffer g % 2
        const int64_t total_chunks = (int64_t)passes * n_chunks;
        const bool resident = n_chunks <= 2;
        __syncthreads();
        if (tid == 0) {
            fence_proxy_async_smem();
            for (int g = 0; g < 2 && g < (resident ? n_chunks : total_chunks); ++g) {
                const int ch = g % n_chunks;
                const int cnt = min(CHUNK_INSTR, D.n_instr - ch * CHUNK_INSTR);
                const uint32_t bytes = (uint32_t)((cnt * 8 + 15) & ~15);
                mbar_expect_tx(&bars[g], bytes);
                bulk_g2s(buf[g], D.tape + (int64_t)ch * CHUNK_INSTR, bytes, &bars[g]);
            }
        }
        int64_t g = 0;   // global chunk counter
        for (int pass = 0; pass < passes && !failed; ++pass) {
            const int64_t i = first + (int64_t)pass * T + tid;
            const bool valid = i < last;
            // zero roots, then the prologue
            const int base_roots = 5 + 4 * D.order + 3 * (D.order - 1);
            for (int r = 0; r < 2 * D.n_roots; ++r) S[base_roots + r] = 0.0f;
            prologue(S, D, A, valid ? i : first, inst);
            // tape
            for (int ch = 0; ch < n_chunks; ++ch, ++g) {
                const int b = resident ? ch : (int)(g & 1);
                if (!resident || pass == 0) {
                    const bool ok = mbar_wait_bounded(&bars[b], phase[b] & 1u, WAIT_LIMIT);
                    // block-uniform decision: every thread takes the same branch
                    if (__syncthreads_or(!ok)) {
                        failed = true;
                        if (tid == 0 && A.status) atomicExch(A.status, DEV_ST_TIMEOUT);
                        if (ok) ++phase[b];
                        break;
                    }
                    ++phase[b];
                }
                const int cnt = min(CHUNK_INSTR, D.n_instr - ch * CHUNK_INSTR);
                run_chunk(S, buf[b], cnt, D);
                if (!resident) {
                    __syncthreads();    // everybody is done with buffer b
                    const int64_t nxt = g + 2;
                    if (tid == 0 && nxt < total_chunks) {
                        fence_proxy_async_smem();
                        const int nch = (int)(nxt % n_chunks);
                        const int ncnt = min(CHUNK_INSTR, D.n_instr - nch * CHUNK_INSTR);
                        const uint32_t bytes = (uint32_t)((ncnt * 8 + 15) & ~15);
                        mbar_expect_tx(&bars[b], bytes);
                        bulk_g2s(buf[b], D.tape + (int64_t)nch * CHUNK_INSTR, bytes, &bars[b]);
                    }
                }
            }
            if (failed) break;
            // epilogue: weighted roots
            float hsum = 0.0f;
            for (int r = 0; r < D.n_roots; ++r) {
                const uint32_t rt = __ldg(D.roots + 2 * r), rs = __ldg(D.roots + 2 * r + 1);
                const int n = (int)(rt & 255u);
                const int dkr = (int)((rt >> 24) & 255u);
                const float J = S[D.n_slots + n - 1];
                float fre = valid ? S[rs & 0xFFFFu] * J : 0.0f;
                float fim = valid ? S[rs >> 16] * J : 0.0f;
                if (!dkr) hsum += fabsf(fre) + fabsf(fim);
                if (A.per_sample_f && valid) {
                    const int64_t o = (((int64_t)inst * A.r_max + r) * 2) * A.n_per_inst + i;
                    A.per_sample_f[o] = fre;
                    A.per_sample_f[o + A.n_per_inst] = fim;
                }
                float v[4] = {fre, fre * fre, fim, fim * fim};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
#pragma unroll
                    for (int off = 16; off > 0; off >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], off);
                }
                if (lane == 0) {
                    double *wa = acc + (size_t)warp * racc * 2;
#pragma unroll
                    for (int q = 0; q < 4; ++q) neumaier(wa[(r * 4 + q) * 2], wa[(r * 4 + q) * 2 + 1], (double)v[q]);
                }
            }
            if (D.hist && valid && !D.points) {
                const double h = (double)hsum * (double)hsum;
                for (int d = 0; d < D.dim; ++d) {
                    const int bin = __float_as_int(S[D.n_slots + D.order + d]);
                    atomicAdd(D.hist + (int64_t)d * D.n_bins + bin, h);
                }
            }
        }
        __syncthreads();
        if (!failed) {
            // combine warps in a fixed order into the tile partials
            for (int k = tid; k < D.n_roots * 4; k += T) {
                double s = 0.0, c = 0.0;
                for (int wp = 0; wp < T / 32; ++wp) {
                    const double *wa = acc + (size_t)wp * racc * 2;
                    neumaier(s, c, wa[k * 2]);
                    neumaier(s, c, wa[k * 2 + 1]);
                }
                const int r = k / 4, q = k % 4;   // q: 0 re sum, 1 re sumsq, 2 im sum, 3 im sumsq
                const int64_t o = (((int64_t)inst * A.tiles_per_inst + tile) * A.r_max + r) * 4;
                A.partials[o + (q / 2) * 2 + (q % 2)] = s + c;
            }
            // roots beyond this graph's count are zero
            for (int k = D.n_roots * 4 + tid; k < A.r_max * 4; k += T) {
                const int64_t o = ((int64_t)inst * A.tiles_per_inst + tile) * A.r_max * 4;
                A.partials[o + k] = 0.0;
            }
        }
        __syncthreads();
    }
    if (failed && tid == 0) {
        // bounded wait for copies still in flight into this CTA's buffers
        for (int b = 0; b < 2; ++b) (void)mbar_wait_bounded(&bars[b], phase[b] & 1u, WAIT_LIMIT);
    }
}

template <int T>
fd_status launch_eval(const EvalArgs &args, cudaStream_t stream, int items) {
    const SmemLayout L = smem_layout(T, args.slots_total, args.r_max);
    int dev = 0;
    FD_CHECK_CUDA(cudaGetDevice(&dev));
    int max_smem = 0, n_sm = 0;
    FD_CHECK_CUDA(cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    FD_CHECK_CUDA(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
    if (L.total > max_smem)
        return fd::set_error(FD_ENOTSUP, "graph needs " + std::to_string(L.total) +
                                             " bytes of shared memory per CTA (limit " +
                                             std::to_string(max_smem) + ")");
    FD_CHECK_CUDA(cudaFuncSetAttribute(integrand_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, L.total));
    int per_sm = 0;
    FD_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, integrand_kernel<T>, T, L.total));
    per_sm = std::max(per_sm, 1);
    const int grid = std::min(items, n_sm * per_sm);
    integrand_kernel<T><<<grid, T, L.total, stream>>>(args);
    FD_CHECK_CUDA(cudaGetLastError());
    return FD_OK;
}

}  // namespace

extern "C" int64_t fd_partials_count(int32_t n_inst, int32_t r_max, int64_t n_per_inst) {
    if (n_inst <= 0 || r_max <= 0 || n_per_inst <= 0) return 0;
    const int64_t tiles = (n_per_inst + FD_TILE_SAMPLES - 1) / FD_TILE_SAMPLES;
    return (int64_t)n_inst * tiles * r_max * 4;
}

namespace {
// Shared body of the evaluation entry points: validate, build the launch
// descriptors and launch the integrand kernel.  `status` is the device word a
// kernel sets when a bounded wait gives up (may be null).
fd_status eval_impl(const fd_graph *const *graphs, int32_t n_graphs, const fd_params *params,
                    const int32_t *graph_of_inst, int32_t n_inst, fd_vegas *const *maps,
                    const float *points, const float *point_w, uint64_t seed, uint64_t iter,
                    int64_t n_per_inst, double *partials, float *per_sample_f, int *status,
                    cudaStream_t stream) {
    FD_REQUIRE(graphs && n_graphs > 0, "graphs must be a non-empty array");
    FD_REQUIRE(params && graph_of_inst, "params and graph_of_inst are required");
    FD_REQUIRE(n_inst > 0 && n_inst <= FD_MAX_INST, "n_inst must be in [1, 256]");
    FD_REQUIRE(n_per_inst > 0 && n_per_inst <= (int64_t(1) << 40), "n_per_inst out of range");
    FD_REQUIRE(partials, "partials buffer is required");
    FD_REQUIRE(point_w == nullptr || points != nullptr, "point_w needs points");
    static EvalArgs args;   // large (kernel parameter space); built on the host per call
    args.n_inst = n_inst;
    args.n_per_inst = n_per_inst;
    args.tiles_per_inst = (int32_t)((n_per_inst + FD_TILE_SAMPLES - 1) / FD_TILE_SAMPLES);
    args.seed_lo = (uint32_t)seed;
    args.seed_hi = (uint32_t)(seed >> 32);
    args.iter = (uint32_t)iter;
    args.partials = partials;
    args.per_sample_f = per_sample_f;
    args.status = status;
    int r_max = 0, slots_total = 0, dim_max = 0;
    for (int g = 0; g < n_graphs; ++g) {
        FD_REQUIRE(graphs[g], "null graph handle");
        const TapeHeader &h = graphs[g]->hdr;
        r_max = std::max(r_max, (int)h.n_roots);
        slots_total = std::max(slots_total, (int)(h.n_slots + h.order + h.dim));
        dim_max = std::max(dim_max, (int)h.dim);
    }
    args.r_max = r_max;
    args.slots_total = slots_total;
    args.dim_max = dim_max;
    for (int j = 0; j < n_inst; ++j) {
        const int gi = graph_of_inst[j];
        FD_REQUIRE(gi >= 0 && gi < n_graphs, "graph_of_inst out of range");
        const fd_graph *G = graphs[gi];
        const fd_params &p = params[j];
        FD_REQUIRE(p.order == (int)G->hdr.order, "params.order differs from the graph order");
        FD_REQUIRE(std::isfinite(p.k_ext) && std::isfinite(p.mu) && std::isfinite(p.beta) &&
                       std::isfinite(p.Lambda) && std::isfinite(p.k_cut),
                   "non-finite parameter");
        FD_REQUIRE(p.beta > 0 && p.Lambda > 0 && p.k_cut > 0 && p.k_ext >= 0,
                   "beta, Lambda, k_cut must be positive and k_ext non-negative");
        InstDesc &D = args.inst[j];
        D.tape = G->d_tape;
        D.roots = G->d_roots;
        D.n_instr = (int32_t)G->hdr.n_instr;
        D.n_slots = (int32_t)G->hdr.n_slots;
        D.order = (int32_t)G->hdr.order;
        D.dim = (int32_t)G->hdr.dim;
        D.n_roots = (int32_t)G->hdr.n_roots;
        D.kext = (float)p.k_ext;
        D.mu = (float)p.mu;
        D.beta = (float)p.beta;
        D.Lambda = (float)p.Lambda;
        D.kc = (float)p.k_cut;
        D.edges = nullptr;
        D.hist = nullptr;
        D.n_bins = 1;
        D.points = nullptr;
        D.point_w = nullptr;
        if (points) {
            D.points = points + (int64_t)j * dim_max * n_per_inst;
            D.point_w = point_w ? point_w + (int64_t)j * n_per_inst : nullptr;
        } else if (maps && maps[j]) {
            FD_REQUIRE(maps[j]->dim == D.dim, "VEGAS map dimension differs from the graph dimension");
            D.edges = maps[j]->d_edges32;
            D.hist = maps[j]->d_hist;
            D.n_bins = maps[j]->n_bins;
        }
    }
    const int items = n_inst * args.tiles_per_inst;
    int dev = 0, max_smem = 0;
    FD_CHECK_CUDA(cudaGetDevice(&dev));
    FD_CHECK_CUDA(cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    // widest CTA whose per-sample state fits in shared memory
    if (smem_layout(128, args.slots_total, args.r_max).total <= max_smem)
        return launch_eval<128>(args, stream, items);
    if (smem_layout(64, args.slots_total, args.r_max).total <= max_smem)
        return launch_eval<64>(args, stream, items);
    return launch_eval<32>(args, stream, items);
}
}  // namespace

extern "C" fd_status fd_integrand_eval(const fd_graph *const *graphs, int32_t n_graphs,
                                       const fd_params *params, const int32_t *graph_of_inst,
                                       int32_t n_inst, fd_vegas *const *maps, const float *points,
                                       const float *point_w, uint64_t seed, uint64_t iter,
                                       int64_t n_per_inst, double *partials, float *per_sample_f,
                                       void *stream) {
    return eval_impl(graphs, n_graphs, params, graph_of_inst, n_inst, maps, points, point_w, seed, iter,
                     n_per_inst, partials, per_sample_f, fd::device_status_word(), (cudaStream_t)stream);
}

// ---- fd_accumulate ---------------------------------------------------------------
namespace {
__global__ void accumulate_kernel(const double *partials, int n_inst, int r_max, int tiles,
                                  int64_t n, double *out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;   // (inst, r, c)
    if (k >= n_inst * r_max * 2) return;
    const int inst = k / (r_max * 2), rc = k % (r_max * 2), r = rc / 2, c = rc % 2;
    double s = 0.0, sc = 0.0, q = 0.0, qc = 0.0;
    for (int t = 0; t < tiles; ++t) {
        const double *p = partials + (((int64_t)inst * tiles + t) * r_max + r) * 4 + c * 2;
        neumaier(s, sc, p[0]);
        neumaier(q, qc, p[1]);
    }
    s += sc;
    q += qc;
    const double mean = s / (double)n;
    double var = 0.0;
    if (n > 1) var = fmax((q - s * mean) / (double)(n - 1), 0.0) / (double)n;
    out[(((int64_t)inst * r_max + r) * 2 + c) * 2] = mean;
    out[(((int64_t)inst * r_max + r) * 2 + c) * 2 + 1] = var;
}
}  // namespace

extern "C" fd_status fd_accumulate(const double *partials, int32_t n_inst, int32_t r_max,
                                   int64_t n_per_inst, double *out, void *stream) {
    FD_REQUIRE(partials && out, "partials and out are required");
    FD_REQUIRE(n_inst > 0 && r_max > 0 && n_per_inst > 0, "sizes must be positive");
    const int tiles = (int)((n_per_inst + FD_TILE_SAMPLES - 1) / FD_TILE_SAMPLES);
    const int total = n_inst * r_max * 2;
    accumulate_kernel<<<(total + 127) / 128, 128, 0, (cudaStream_t)stream>>>(partials, n_inst, r_max, tiles,
                                                                          n_per_inst, out);
    FD_CHECK_CUDA(cudaGetLastError());
    return FD_OK;
}

// ---- evaluation without device allocation ---------------------------------------
// Callers that cannot allocate device memory themselves (a host process whose
// allocations must all be made up front, a CUDA-graph replay that may not add
// new memory, or a caller without a device allocator in reach) still need
// the tile partial sums between the two reduction passes.  This variant keeps
// them in a fixed array of this library instead.  The array lives in every
// device's global memory for as long as the library stays loaded.
namespace {
__device__ __align__(256) double g_noalloc_partials[FD_NOALLOC_MAX_PARTIALS];

struct NoallocDevice {
    bool ready = false;
    double *partials = nullptr;   // device address of g_noalloc_partials on that device
};
NoallocDevice g_noalloc_dev[64];
std::mutex g_noalloc_mu;

// Once per device, with that device current: resolve the array's device
// address (its host-side name is only a stand-in and must never reach a kernel).
fd_status noalloc_setup(double **out) {
    int dev = 0;
    FD_CHECK_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fd::set_error(FD_ENOTSUP, "device index beyond 63");
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    NoallocDevice &d = g_noalloc_dev[dev];
    if (!d.ready) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
        if (e != cudaSuccess) return fd::cuda_error(e, "cudaGetSymbolAddress(g_noalloc_partials)");
        d.partials = static_cast<double *>(p);
        d.ready = true;
    }
    *out = d.partials;
    return FD_OK;
}
}  // namespace

extern "C" fd_status fd_integrand_eval_stats_noalloc(
    const fd_graph *const *graphs, int32_t n_graphs, const fd_params *params, const int32_t *graph_of_inst,
    int32_t n_inst, fd_vegas *const *maps, const float *points, const float *point_w, uint64_t seed,
    uint64_t iter, int64_t n_per_inst, double *out, float *per_sample_f, void *stream) {
    FD_REQUIRE(graphs && n_graphs > 0, "graphs must be a non-empty array");
    FD_REQUIRE(out, "out is required");
    FD_REQUIRE(n_inst > 0 && n_inst <= FD_MAX_INST, "n_inst must be in [1, 256]");
    FD_REQUIRE(n_per_inst > 0 && n_per_inst <= (int64_t(1) << 40), "n_per_inst out of range");
    int r_max = 0;
    for (int g = 0; g < n_graphs; ++g) {
        FD_REQUIRE(graphs[g], "null graph handle");
        r_max = std::max(r_max, (int)graphs[g]->hdr.n_roots);
    }
    const int64_t need = fd_partials_count(n_inst, r_max, n_per_inst);
    if (need > (int64_t)FD_NOALLOC_MAX_PARTIALS)
        return fd::set_error(FD_EINVAL, "request needs " + std::to_string(need) +
                                            " partial sums; the fixed array holds " +
                                            std::to_string((long long)FD_NOALLOC_MAX_PARTIALS) +
                                            " (use fd_integrand_eval with a caller buffer)");
    double *partials = nullptr;
    fd_status st = noalloc_setup(&partials);
    if (st != FD_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    // every byte 0xFF is a NaN double: a tile the kernel failed to write shows up
    // as NaN in `out` instead of a stale value from an earlier call
    FD_CHECK_CUDA(cudaMemsetAsync(partials, 0xFF, (size_t)need * sizeof(double), s));
    st = eval_impl(graphs, n_graphs, params, graph_of_inst, n_inst, maps, points, point_w, seed, iter, n_per_inst,
                   partials, per_sample_f, nullptr, s);
    if (st != FD_OK) return st;
    return fd_accumulate(partials, n_inst, r_max, n_per_inst, out, stream);
}
