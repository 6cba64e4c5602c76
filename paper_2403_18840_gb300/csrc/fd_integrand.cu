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
//  * persistent CTAs walk work items = (instance, tile of fd_tile_samples(n)
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
#include <atomic>
#include <mutex>
#include <string>
#include <vector>

#include "fd_internal.cuh"

namespace {

constexpr int CHUNK_INSTR = FD_CHUNK_WORDS;           // 8 KB per tape buffer
constexpr int CHUNK_BYTES = CHUNK_INSTR * 8;
constexpr uint32_t WAIT_LIMIT = 1u << 24;             // polls before a tape wait gives up
constexpr int NK = FD_MAX_ORDER;                      // loop momenta / interaction lines held in registers

struct SmemLayout {
    int tape0, tape1, bars, acc, slots, total;   // byte offsets in dynamic shared memory
};

__host__ __device__ inline SmemLayout smem_layout(int threads, int P, int slots_total, int r_max) {
    SmemLayout L;
    L.tape0 = 0;
    L.tape1 = CHUNK_BYTES;
    L.bars = 2 * CHUNK_BYTES;
    L.acc = L.bars + 16;
    const int nwarps = threads / 32;
    L.slots = L.acc + nwarps * r_max * 4 * 2 * 8;            // (sum, sumsq) x (re, im) x (value, comp)
    L.slots = (L.slots + 15) & ~15;
    L.total = L.slots + slots_total * threads * P * 4;
    return L;
}

// per-sample slots in shared memory: [slot][thread][P] FP32
template <int T, int P>
struct Slots {
    float *base;
    __device__ __forceinline__ float *at(uint32_t s) const { return base + (size_t)s * (T * P); }
    __device__ __forceinline__ void load(uint32_t s, float (&v)[P]) const {
        if constexpr (P == 2) {
            const float2 f = *reinterpret_cast<const float2 *>(at(s));
            v[0] = f.x;
            v[1] = f.y;
        } else {
#pragma unroll
            for (int p = 0; p < P; ++p) v[p] = at(s)[p];
        }
    }
    __device__ __forceinline__ void store(uint32_t s, const float (&v)[P]) const {
        if constexpr (P == 2) {
            *reinterpret_cast<float2 *>(at(s)) = make_float2(v[0], v[1]);
        } else {
#pragma unroll
            for (int p = 0; p < P; ++p) at(s)[p] = v[p];
        }
    }
    __device__ __forceinline__ void store1(uint32_t s, int p, float v) const { at(s)[p] = v; }
};

// register-resident per-sample variables
template <int P>
struct Vars {
    float kx[NK][P], ky[NK][P], kz[NK][P];     // loop momenta k_1..k_N: grid parts
    float kxl[NK][P], kyl[NK][P], kzl[NK][P];  // and remainders
    float tl[NK][P];                           // remainders of the times of interaction lines 0..N-1 (hi: slots 2..)
    float re[P], im[P], hsum[P];               // root accumulator and |f| sum for VEGAS
};

template <int P>
__device__ __forceinline__ float pick(const float (&a)[NK][P], uint32_t idx, int p) {
    float r = a[0][p];
#pragma unroll
    for (int j = 1; j < NK; ++j) r = (idx == (uint32_t)j) ? a[j][p] : r;
    return r;
}

__device__ __forceinline__ uint32_t f_d(uint64_t w) { return (uint32_t)(w >> 6) & 16383u; }
__device__ __forceinline__ uint32_t f_a(uint64_t w) { return (uint32_t)(w >> 20) & 16383u; }
__device__ __forceinline__ uint32_t f_b(uint64_t w) { return (uint32_t)(w >> 34) & 16383u; }

// signed momentum sums from a 2-bit-per-variable mask, grid parts (h) and
// remainders (l); k_ext is (0, 0, kext + kext_l)
template <int P>
__device__ __forceinline__ void momentum(const Vars<P> &V, uint32_t mask, const InstDesc &D, float (&h)[3][P],
                                         float (&l)[3][P], float &ks) {
    float cf[NK + 1];
#pragma unroll
    for (int j = 0; j <= NK; ++j) cf[j] = (float)(((int)(mask << (30 - 2 * j))) >> 30);   // signed 2-bit field
    ks = cf[0];
#pragma unroll
    for (int p = 0; p < P; ++p) {
        float x = 0.0f, y = 0.0f, z = cf[0] * D.kext, xl = 0.0f, yl = 0.0f, zl = cf[0] * D.kext_l;
#pragma unroll
        for (int j = 0; j < NK; ++j) {
            x = fmaf(cf[j + 1], V.kx[j][p], x);                 // exact: grid values, coefficients 0, +-1
            y = fmaf(cf[j + 1], V.ky[j][p], y);
            z = fmaf(cf[j + 1], V.kz[j][p], z);
            xl = fmaf(cf[j + 1], V.kxl[j][p], xl);
            yl = fmaf(cf[j + 1], V.kyl[j][p], yl);
            zl = fmaf(cf[j + 1], V.kzl[j][p], zl);
        }
        h[0][p] = x;
        h[1][p] = y;
        h[2][p] = z;
        l[0][p] = xl;
        l[1][p] = yl;
        l[2][p] = zl;
    }
}

// G0 and V Taylor families of one leaf instruction (g_family / v_family),
// written to the slots d, d + 1, ...
template <int T, int P>
__device__ __forceinline__ void g_leaf(const Slots<T, P> &S, const Vars<P> &V, uint64_t w, const InstDesc &D) {
    const uint32_t d = f_d(w), mask = f_a(w);
    const uint32_t la = (uint32_t)(w >> 34) & 7u, lb = (uint32_t)(w >> 37) & 7u;
    const int M = (int)((w >> 40) & 7u);
    const int dk = (int)((w >> 43) & 1u);
    const bool precise = (w >> FD_LEAF_PRECISE_BIT) & 1u;
    float h[3][P], l[3][P], ks;
    momentum(V, mask, D, h, l, ks);
    float ta[P], tb[P];
    S.load(2 + la, ta);                        // hypercube time of the two lines
    S.load(2 + lb, tb);
#pragma unroll
    for (int p = 0; p < P; ++p) {
        float dxh, dxl;
        fd_time_diff(ta[p], pick(V.tl, la, p), tb[p], pick(V.tl, lb, p), dxh, dxl);
        if (precise) {
            g_family_df(h[0][p], h[1][p], h[2][p], FdDF{l[0][p], 0.0f}, FdDF{l[1][p], 0.0f}, FdDF{l[2][p], 0.0f},
                        ks, dxh, dxl, D.beta, D.beta_l, D.mu, D.mu_l, M, dk,
                        [&](int j, float v) { S.store1(d + j, p, v); });
            continue;
        }
        const float eps = fd_eps(h[0][p], h[1][p], h[2][p], l[0][p], l[1][p], l[2][p], D.mu, D.mu_l);
        g_family<float>(eps, h[2][p] + l[2][p], ks, dxh, dxl, D.beta, M, dk,
                        [&](int j, float v) { S.store1(d + j, p, v); });
    }
}

template <int T, int P>
__device__ __forceinline__ void v_leaf(const Slots<T, P> &S, const Vars<P> &V, uint64_t w, const InstDesc &D) {
    const uint32_t d = f_d(w), mask = f_a(w);
    const int L = (int)((w >> 40) & 7u);
    const int dk = (int)((w >> 43) & 1u);
    float h[3][P], l[3][P], ks;
    momentum(V, mask, D, h, l, ks);
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const float qx = h[0][p] + l[0][p], qy = h[1][p] + l[1][p], qz = h[2][p] + l[2][p];
        const float q2 = fmaf(qx, qx, fmaf(qy, qy, qz * qz));
        v_family<float>(q2, qz, ks, D.Lambda, L, dk, [&](int j, float v) { S.store1(d + j, p, v); });
    }
}

// Root r is complete for the current samples: weight, write, reduce, reset.
template <int T, int P>
__device__ __forceinline__ void flush_root(const Slots<T, P> &S, Vars<P> &V, uint32_t r, const InstDesc &D,
                                           const EvalArgs &A, double *acc, int inst, const int64_t (&idx)[P],
                                           const bool (&valid)[P]) {
    const uint32_t rt = __ldg(D.roots + 2 * r);
    const uint32_t n = rt & 255u;
    const bool dkr = ((rt >> 24) & 255u) != 0;
    float jw[P];
    S.load(D.n_slots + D.dim + n - 1, jw);     // weight of the roots of order n
    float v[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const float J = jw[p];
        const float fre = valid[p] ? V.re[p] * J : 0.0f;
        const float fim = valid[p] ? V.im[p] * J : 0.0f;
        V.re[p] = 0.0f;
        V.im[p] = 0.0f;
        if (!dkr) V.hsum[p] += fabsf(fre) + fabsf(fim);
        if (A.per_sample_f && valid[p]) {
            const int64_t o = (((int64_t)D.id * A.r_max + r) * 2) * A.n_per_inst + idx[p];
            A.per_sample_f[o] = fre;
            A.per_sample_f[o + A.n_per_inst] = fim;
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
        double *wa = acc + (size_t)(threadIdx.x >> 5) * A.r_max * 8;
#pragma unroll
        for (int q = 0; q < 4; ++q) neumaier(wa[(r * 4 + q) * 2], wa[(r * 4 + q) * 2 + 1], (double)v[q]);
    }
}

template <int T, int P>
__device__ __forceinline__ void run_chunk(const Slots<T, P> &S, Vars<P> &V, const uint64_t *code, int cnt,
                                          const InstDesc &D, const EvalArgs &A, double *acc, int inst,
                                          const int64_t (&idx)[P], const bool (&valid)[P]) {
    for (int k = 0; k < cnt; ++k) {
        const uint64_t w = code[k];
        const uint32_t op = (uint32_t)w & 63u;
        if (op == OP_BUNDLE) {
            // independent FMAs: every operand is loaded before any result is stored
            const int n = (int)((w >> 6) & 15u);
            const uint64_t *q = code + k + 1;
            float a[FD_MAX_BUNDLE][P], b[FD_MAX_BUNDLE][P], c[FD_MAX_BUNDLE][P];
            uint32_t dst[FD_MAX_BUNDLE];
#pragma unroll
            for (int j = 0; j < FD_MAX_BUNDLE; ++j) {
                if (j < n) {
                    const uint2 ww = *reinterpret_cast<const uint2 *>(q + j);
                    dst[j] = ww.x & 0xFFFFu;
                    S.load(ww.x >> 16, a[j]);
                    S.load(ww.y & 0xFFFFu, b[j]);
                    S.load(ww.y >> 16, c[j]);
                }
            }
#pragma unroll
            for (int j = 0; j < FD_MAX_BUNDLE; ++j) {
                if (j < n) {
#pragma unroll
                    for (int p = 0; p < P; ++p) a[j][p] = fmaf(a[j][p], b[j][p], c[j][p]);
                    S.store(dst[j], a[j]);
                }
            }
            k += n;
            continue;
        }
        switch (op) {
            case OP_GLEAF:
                g_leaf(S, V, w, D);
                break;
            case OP_VLEAF:
                v_leaf(S, V, w, D);
                break;
            case OP_RACC: {
                float a[P], tl[P];
                S.load(f_a(w), a);
                const uint32_t line = f_b(w);
                S.load(2 + line, tl);
#pragma unroll
                for (int p = 0; p < P; ++p) {
                    float sn = 0.0f, cs = 1.0f;
                    if (line) sincospif(tl[p], &sn, &cs);
                    V.re[p] = fmaf(a[p], cs, V.re[p]);
                    V.im[p] = fmaf(a[p], sn, V.im[p]);
                }
                break;
            }
            case OP_RFLUSH:
                flush_root<T, P>(S, V, f_d(w), D, A, acc, inst, idx, valid);
                break;
            case OP_CONST: {
                float c[P];
#pragma unroll
                for (int p = 0; p < P; ++p) c[p] = __uint_as_float((uint32_t)(w >> 32));
                S.store(f_d(w), c);
                break;
            }
            case OP_NOP:
                break;
            default:
                return;   // OP_END
        }
    }
}

// Sample generation: Philox -> uniforms -> VEGAS (or given points) -> loop
// momenta, times, phases and per-order weights in registers; VEGAS bins in
// the slots [n_slots, n_slots + dim).
template <int T, int P>
__device__ __forceinline__ void prologue(const Slots<T, P> &S, Vars<P> &V, const InstDesc &D, const EvalArgs &A,
                                         const int64_t (&idx)[P], int inst, uint32_t iter) {
    const int N = D.order, dim = D.dim;
    float one[P], zero[P];
#pragma unroll
    for (int p = 0; p < P; ++p) {
        one[p] = 1.0f;
        zero[p] = 0.0f;
    }
    S.store(0, zero);
    S.store(1, one);
    S.store(2, zero);                           // time of interaction line 0
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const int64_t i = idx[p];
        FdDF x[FD_MAX_DIM];
        float wgt = 1.0f;
        if (D.points) {
#pragma unroll
            for (int d = 0; d < FD_MAX_DIM; ++d)
                if (d < dim) x[d] = FdDF{D.points[(int64_t)d * A.n_per_inst + i], 0.0f};
            wgt = D.point_w ? D.point_w[i] : 1.0f;
        } else {
            const uint32_t c0 = (uint32_t)(uint64_t)i, c1 = (uint32_t)((uint64_t)i >> 32);
#pragma unroll
            for (int blk = 0; blk < (FD_MAX_DIM + 3) / 4; ++blk) {
                if (4 * blk < dim) {
                    const u32x4 r = philox4x32_10(
                        u32x4{c0, c1, iter, ((uint32_t)D.id << 8) | (uint32_t)blk}, A.seed_lo, A.seed_hi);
                    const uint32_t wv[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        if (4 * blk + q < FD_MAX_DIM) x[4 * blk + q] = FdDF{word_to_uniform(wv[q]), 0.0f};
                }
            }
        }
        float jd[FD_MAX_DIM];
#pragma unroll
        for (int d = 0; d < FD_MAX_DIM; ++d) {
            jd[d] = 1.0f;
            if (d < dim && D.edges) {
                const int bin = fd_vegas_df(x[d].hi, D.n_bins, D.edges + (int64_t)d * (D.n_bins + 1), x[d], jd[d]);
                S.store1(D.n_slots + d, p, __int_as_float(bin));
            }
        }
        const float g = D.grid, ginv = 1.0f / D.grid;
        float jac = wgt;
        V.tl[0][p] = 0.0f;
#pragma unroll
        for (int j = 0; j < NK; ++j) {
            V.kx[j][p] = V.ky[j][p] = V.kz[j][p] = 0.0f;
            V.kxl[j][p] = V.kyl[j][p] = V.kzl[j][p] = 0.0f;
            if (j >= 1) V.tl[j][p] = 0.0f;
            const int jj = j + 1;                       // loop momentum k_jj
            if (jj <= N) {
                const int c0 = (jj == 1) ? 0 : 4 * jj - 5;
                float kh[3], kl[3];
                const float r =
                    fd_loop_momentum(x[c0], x[c0 + 1], x[c0 + 2], FdDF{D.kc, D.kc_l}, A.sc_tab, g, ginv, kh, kl);
                V.kx[j][p] = kh[0];
                V.ky[j][p] = kh[1];
                V.kz[j][p] = kh[2];
                V.kxl[j][p] = kl[0];
                V.kyl[j][p] = kl[1];
                V.kzl[j][p] = kl[2];
                jac *= D.kc * r * r * FD_INV_2PI2;
                jac *= jd[c0] * jd[c0 + 1] * jd[c0 + 2];   // 1 without a map
                if (jj >= 2) {
                    // time of interaction line jj - 1
                    S.store1(2 + jj - 1, p, x[4 * jj - 2].hi);
                    V.tl[jj - 1][p] = x[4 * jj - 2].lo;
                    jac *= D.beta;
                    jac *= jd[4 * jj - 2];
                }
                S.store1(D.n_slots + D.dim + j, p, jac);
            }
        }
        V.re[p] = 0.0f;
        V.im[p] = 0.0f;
        V.hsum[p] = 0.0f;
    }
}

template <int T, int P>
__global__ void __launch_bounds__(T) integrand_kernel(const __grid_constant__ EvalArgs A) {
    extern __shared__ __align__(16) unsigned char smem[];
    const SmemLayout L = smem_layout(T, P, A.slots_total, A.r_max);
    uint64_t *buf[2] = {reinterpret_cast<uint64_t *>(smem + L.tape0),
                        reinterpret_cast<uint64_t *>(smem + L.tape1)};
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + L.bars);
    double *acc = reinterpret_cast<double *>(smem + L.acc);
    const int tid = threadIdx.x;
    const Slots<T, P> S{reinterpret_cast<float *>(smem + L.slots) + tid * P};
    const int n_items = A.n_inst * A.tiles_per_inst;
    const int racc = A.r_max * 8;   // doubles per warp

    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_mbarrier_init();
    }
    __syncthreads();
    uint32_t phase[2] = {0u, 0u};
    bool pending[2] = {false, false};   // (thread 0) a bulk copy into buffer b has not been waited for
    bool failed = false;
    Vars<P> V;
    const uint32_t iter = A.iter + (A.iter_dev ? *A.iter_dev : 0u);
    __shared__ int next_item;

    for (;;) {
        // dynamic work queue: heaviest instances first, then their tiles
        if (tid == 0) next_item = (int)atomicAdd(A.queue, 1ull);
        __syncthreads();
        const int item = next_item;
        if (item >= n_items || failed) break;
        const int inst = A.perm[item / A.tiles_per_inst];
        const int tile = item % A.tiles_per_inst;
        const InstDesc &D = A.inst[inst];
        const int n_chunks = (D.n_instr + CHUNK_INSTR - 1) / CHUNK_INSTR;
        for (int k = tid; k < (T / 32) * racc; k += T) acc[k] = 0.0;
        const int64_t first = (int64_t)tile * A.tile;
        const int64_t last = min(first + A.tile, A.n_per_inst);
        const int passes = (int)((last - first + T * P - 1) / (T * P));
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
                pending[g] = true;
            }
        }
        int64_t g = 0;
        for (int pass = 0; pass < passes && !failed; ++pass) {
            int64_t idx[P];
            bool valid[P];
#pragma unroll
            for (int p = 0; p < P; ++p) {
                const int64_t i = first + (int64_t)pass * T * P + (int64_t)p * T + tid;
                valid[p] = i < last;
                idx[p] = valid[p] ? i : first;
            }
            prologue<T, P>(S, V, D, A, idx, inst, iter);
            for (int ch = 0; ch < n_chunks; ++ch, ++g) {
                const int b = resident ? ch : (int)(g & 1);
                if (!resident || pass == 0) {
                    const bool ok = mbar_wait_bounded(&bars[b], phase[b] & 1u, A.wait_polls);
                    if (ok) {
                        ++phase[b];
                        pending[b] = false;
                    }
                    // block-uniform decision: every thread takes the same branch
                    if (__syncthreads_or(!ok)) {
                        failed = true;
                        if (tid == 0 && A.status) atomicExch(A.status, DEV_ST_TIMEOUT);
                        break;
                    }
                }
                const int cnt = min(CHUNK_INSTR, D.n_instr - ch * CHUNK_INSTR);
                run_chunk<T, P>(S, V, buf[b], cnt, D, A, acc, inst, idx, valid);
                if (!resident) {
                    __syncthreads();
                    const int64_t nxt = g + 2;
                    if (tid == 0 && nxt < total_chunks) {
                        fence_proxy_async_smem();
                        const int nch = (int)(nxt % n_chunks);
                        const int ncnt = min(CHUNK_INSTR, D.n_instr - nch * CHUNK_INSTR);
                        const uint32_t bytes = (uint32_t)((ncnt * 8 + 15) & ~15);
                        mbar_expect_tx(&bars[b], bytes);
                        bulk_g2s(buf[b], D.tape + (int64_t)nch * CHUNK_INSTR, bytes, &bars[b]);
                        pending[b] = true;
                    }
                }
            }
            if (failed) break;
            if (A.abs_f) {
#pragma unroll
                for (int p = 0; p < P; ++p)
                    if (valid[p])
                        A.abs_f[(int64_t)D.id * A.n_per_inst + idx[p]] = isfinite(V.hsum[p]) ? V.hsum[p] : 0.0f;
            }
            if (D.hist && !D.points) {
#pragma unroll
                for (int p = 0; p < P; ++p) {
                    if (!valid[p]) continue;
                    const double h = (double)V.hsum[p] * (double)V.hsum[p];
                    for (int d = 0; d < D.dim; ++d) {
                        const int bin = __float_as_int(S.at(D.n_slots + d)[p]);
                        atomicAdd(D.hist + (int64_t)d * D.n_bins + bin, h);
                    }
                }
            }
        }
        __syncthreads();
        if (!failed) {
            for (int k = tid; k < D.n_roots * 4; k += T) {
                double s = 0.0, c = 0.0;
                for (int wp = 0; wp < T / 32; ++wp) {
                    const double *wa = acc + (size_t)wp * racc;
                    neumaier(s, c, wa[k * 2]);
                    neumaier(s, c, wa[k * 2 + 1]);
                }
                const int r = k / 4, q = k % 4;   // q: 0 re sum, 1 re sumsq, 2 im sum, 3 im sumsq
                const int64_t o = (((int64_t)D.id * A.tiles_per_inst + tile) * A.r_max + r) * 4;
                A.partials[o + q] = s + c;
            }
            for (int k = D.n_roots * 4 + tid; k < A.r_max * 4; k += T) {
                const int64_t o = ((int64_t)D.id * A.tiles_per_inst + tile) * A.r_max * 4;
                A.partials[o + k] = 0.0;
            }
        }
        __syncthreads();
    }
    // after a wait that gave up: thread 0 waits (bounded, at the full limit)
    // for the bulk copies it issued and no wait has consumed, so none is
    // still writing into this CTA's shared memory when it exits
    if (failed && tid == 0) {
        for (int b = 0; b < 2; ++b)
            if (pending[b]) (void)mbar_wait_bounded(&bars[b], phase[b] & 1u, WAIT_LIMIT);
    }
}

template <int T, int P>
fd_status launch_eval(const EvalArgs &args, cudaStream_t stream, int items) {
    const SmemLayout L = smem_layout(T, P, args.slots_total, args.r_max);
    int dev = 0;
    FD_CHECK_CUDA(cudaGetDevice(&dev));
    int max_smem = 0, n_sm = 0;
    FD_CHECK_CUDA(cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    FD_CHECK_CUDA(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
    if (L.total > max_smem)
        return fd::set_error(FD_ENOTSUP, "graph needs " + std::to_string(L.total) +
                                             " bytes of shared memory per CTA (limit " +
                                             std::to_string(max_smem) + ")");
    FD_CHECK_CUDA(cudaFuncSetAttribute(integrand_kernel<T, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, L.total));
    int per_sm = 0;
    FD_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, integrand_kernel<T, P>, T, L.total));
    per_sm = std::max(per_sm, 1);
    const int grid = std::min(items, n_sm * per_sm);
    integrand_kernel<T, P><<<grid, T, L.total, stream>>>(args);
    FD_CHECK_CUDA(cudaGetLastError());
    return FD_OK;
}

}  // namespace

extern "C" fd_status fd_graph_set_launch(fd_graph *g, int32_t threads, int32_t samples_per_thread) {
    FD_REQUIRE(g, "null graph");
    const bool ok = (threads == 0 && samples_per_thread == 0) ||
                    (threads == 128 && samples_per_thread == 2) || (threads == 256 && samples_per_thread == 1) ||
                    (threads == 128 && samples_per_thread == 1) || (threads == 64 && samples_per_thread == 2) ||
                    (threads == 64 && samples_per_thread == 1);
    FD_REQUIRE(ok, "unsupported CTA shape (threads, samples per thread)");
    g->launch_threads = threads;
    g->launch_spt = samples_per_thread;
    return FD_OK;
}

extern "C" int64_t fd_tile_samples(int64_t n_per_inst) {
    int64_t t = 1024;
    while (t < FD_TILE_SAMPLES && t * 4096 < n_per_inst) t *= 2;
    return t;
}

extern "C" int64_t fd_partials_count(int32_t n_inst, int32_t r_max, int64_t n_per_inst) {
    if (n_inst <= 0 || r_max <= 0 || n_per_inst <= 0) return 0;
    const int64_t tl = fd_tile_samples(n_per_inst);
    const int64_t tiles = (n_per_inst + tl - 1) / tl;
    return (int64_t)n_inst * tiles * r_max * 4 + 1;   // + the work-queue counter
}

namespace {
int dev_of_call() {
    int d = -1;
    return cudaGetDevice(&d) == cudaSuccess ? d : -1;
}

// polls before a tape wait of the interpreter gives up (fd_debug_set_wait_polls)
std::atomic<uint32_t> g_wait_polls{WAIT_LIMIT};

// The instance's FP64 parameters as FP32 parts for the kernels' double-float
// kinematics: the grid g is the power of two with max(K_c, k_ext) / g in
// [2^12, 2^13), so every loop-momentum component and k_ext is a multiple of g
// plus a remainder |.| <= g / 2, and sums of up to eight grid parts are exact
// in FP32; mu is split on the grid g^2 (its grid part is exact in FP32 for the
// electron gas, mu = k_F^2 = (K_c / 6)^2), beta and K_c into FP32 roundings
// and remainders.
void set_kinematics(InstDesc &D, const fd_params &p) {
    int e = 0;
    (void)std::frexp(std::max(p.k_cut, p.k_ext), &e);
    const double g = std::ldexp(1.0, e - 13), g2 = g * g;
    const double kh = std::rint(p.k_ext / g) * g;
    const double mh = (double)(float)(std::rint(p.mu / g2) * g2);
    D.grid = (float)g;
    D.kext = (float)kh;
    D.kext_l = (float)(p.k_ext - kh);
    D.mu = (float)mh;
    D.mu_l = (float)(p.mu - mh);
    D.beta = (float)p.beta;
    D.beta_l = (float)(p.beta - (double)D.beta);
    D.kc = (float)p.k_cut;
    D.kc_l = (float)(p.k_cut - (double)D.kc);
    D.Lambda = (float)p.Lambda;
}

// Validation and launch descriptors of an evaluation call (no CUDA work
// beyond device queries): every argument error is reported here, before the
// caller touches any device memory.  `status` is the device word a kernel sets
// when a bounded wait gives up (may be null).
fd_status eval_build(const fd_graph *const *graphs, int32_t n_graphs, const fd_params *params,
                     const int32_t *graph_of_inst, int32_t n_inst, fd_vegas *const *maps,
                     const float *points, const float *point_w, uint64_t seed, uint64_t iter,
                     const uint32_t *iter_dev, int64_t n_per_inst, double *partials, float *per_sample_f,
                     float *abs_f, int *status, EvalArgs &args) {
    FD_REQUIRE(graphs && n_graphs > 0, "graphs must be a non-empty array");
    FD_REQUIRE(params && graph_of_inst, "params and graph_of_inst are required");
    FD_REQUIRE(n_inst > 0 && n_inst <= FD_MAX_INST, "n_inst must be in [1, 256]");
    FD_REQUIRE(n_per_inst > 0 && n_per_inst <= (int64_t(1) << 40), "n_per_inst out of range");
    FD_REQUIRE(partials, "partials buffer is required");
    FD_REQUIRE(point_w == nullptr || points != nullptr, "point_w needs points");
    args.n_inst = n_inst;
    args.n_per_inst = n_per_inst;
    args.tile = fd_tile_samples(n_per_inst);
    args.tiles_per_inst = (int32_t)((n_per_inst + args.tile - 1) / args.tile);
    args.seed_lo = (uint32_t)seed;
    args.seed_hi = (uint32_t)(seed >> 32);
    args.iter = (uint32_t)iter;
    args.wait_polls = g_wait_polls.load();
    args.iter_dev = iter_dev;
    args.partials = partials;
    args.per_sample_f = per_sample_f;
    args.abs_f = abs_f;
    args.status = status;
    int r_max = 0, slots_total = 0, dim_max = 0;
    for (int g = 0; g < n_graphs; ++g) {
        FD_REQUIRE(graphs[g], "null graph handle");
        const TapeHeader &h = graphs[g]->hdr;
        r_max = std::max(r_max, (int)h.n_roots);
        slots_total = std::max(slots_total, (int)(h.n_slots + h.dim + h.order));
        dim_max = std::max(dim_max, (int)h.dim);
    }
    args.r_max = r_max;
    args.slots_total = slots_total;
    args.dim_max = dim_max;
    args.hist_smem = 0;     // the specialised launcher sets its own
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
        set_kinematics(D, p);
        D.id = j;
        D.edges = nullptr;
        D.hist = nullptr;
        D.n_bins = 1;
        D.points = nullptr;
        D.point_w = nullptr;
        if (points) {
            D.points = points + (int64_t)j * dim_max * n_per_inst;
            D.point_w = point_w ? point_w + (int64_t)j * n_per_inst : nullptr;
        }
        if (maps && maps[j]) {
            // given points are the map's input coordinates; only drawn samples adapt the grid
            FD_REQUIRE(maps[j]->dim == D.dim, "VEGAS map dimension differs from the graph dimension");
            D.edges = maps[j]->d_edges32;
            D.hist = points ? nullptr : maps[j]->d_hist;
            D.n_bins = maps[j]->n_bins;
        }
    }
    args.queue = reinterpret_cast<unsigned long long *>(
        partials + fd_partials_count(n_inst, r_max, n_per_inst) - 1);
    for (int g = 0; g < n_graphs; ++g)
        if (graphs[g]->jit_enabled && graphs[g]->jit_kernel)
            FD_REQUIRE(graphs[g]->device == dev_of_call(), "graph belongs to another device");
    return fd::sc_table(&args.sc_tab);
}

// Launches of a built call: instances whose graph has a specialised kernel
// run as one launch per graph (stream-ordered, so they can share the work
// counter); the rest go through the interpreter in one launch.  The
// descriptors live in per-host-thread storage, so calls from several host
// threads do not share them.
fd_status eval_run(const fd_graph *const *graphs, int32_t n_graphs, const int32_t *graph_of_inst, EvalArgs &args,
                   cudaStream_t stream) {
    const int32_t n_inst = args.n_inst;
    bool any_jit = false;
    for (int g = 0; g < n_graphs; ++g) any_jit = any_jit || (graphs[g]->jit_enabled && graphs[g]->jit_kernel);
    if (any_jit) {
        static thread_local EvalArgs sub;
        std::vector<int> rest;
        for (int g = 0; g < n_graphs; ++g) {
            std::vector<int> members;
            for (int j = 0; j < n_inst; ++j)
                if (graph_of_inst[j] == g) members.push_back(j);
            if (members.empty()) continue;
            const fd_graph *G = graphs[g];
            if (!(G->jit_enabled && G->jit_kernel)) {
                rest.insert(rest.end(), members.begin(), members.end());
                continue;
            }
            sub = args;
            sub.n_inst = (int32_t)members.size();
            for (size_t k = 0; k < members.size(); ++k) {
                sub.inst[k] = args.inst[members[k]];
                sub.perm[k] = (uint8_t)k;
            }
            FD_CHECK_CUDA(cudaMemsetAsync(sub.queue, 0, sizeof(unsigned long long), stream));
            const fd_status st = jit_launch(G, sub, stream);
            if (st != FD_OK) return st;
        }
        if (rest.empty()) return FD_OK;
        sub = args;
        sub.n_inst = (int32_t)rest.size();
        for (size_t k = 0; k < rest.size(); ++k) sub.inst[k] = args.inst[rest[k]];
        args = sub;
    }
    const int items = args.n_inst * args.tiles_per_inst;
    // instances in decreasing graph order (cost): longest-processing-time first
    {
        int k = 0;
        for (int o = FD_MAX_ORDER; o >= 1; --o)
            for (int j = 0; j < args.n_inst; ++j)
                if (args.inst[j].order == o) args.perm[k++] = (uint8_t)j;
    }
    FD_CHECK_CUDA(cudaMemsetAsync(args.queue, 0, sizeof(unsigned long long), stream));
    int dev = 0, max_smem = 0;
    FD_CHECK_CUDA(cudaGetDevice(&dev));
    FD_CHECK_CUDA(cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    // CTA shape: the first graph's preference when it fits, otherwise the shape
    // with the most samples in flight per SM (then the most warps)
    const int pref_t = graphs[0]->launch_threads, pref_p = graphs[0]->launch_spt;
    struct Shape { int t, p; };
    const Shape shapes[] = {{128, 2}, {256, 1}, {128, 1}, {64, 2}, {64, 1}};
    auto fits = [&](int t, int p) { return smem_layout(t, p, args.slots_total, args.r_max).total <= max_smem; };
    int bt = 0, bp = 0;
    if (pref_t && fits(pref_t, pref_p)) {
        bt = pref_t;
        bp = pref_p;
    } else {
        long best = -1;
        for (const Shape &sh : shapes) {
            if (!fits(sh.t, sh.p)) continue;
            const int per_cta = smem_layout(sh.t, sh.p, args.slots_total, args.r_max).total;
            const long ctas = std::max(1, (228 * 1024) / per_cta);
            const long score = ctas * sh.t * sh.p * 1000 + ctas * sh.t;
            if (score > best) {
                best = score;
                bt = sh.t;
                bp = sh.p;
            }
        }
    }
    if (bt == 128 && bp == 2) return launch_eval<128, 2>(args, stream, items);
    if (bt == 256 && bp == 1) return launch_eval<256, 1>(args, stream, items);
    if (bt == 128 && bp == 1) return launch_eval<128, 1>(args, stream, items);
    if (bt == 64 && bp == 2) return launch_eval<64, 2>(args, stream, items);
    if (bt == 64 && bp == 1) return launch_eval<64, 1>(args, stream, items);
    return fd::set_error(FD_ENOTSUP, "per-sample state of " + std::to_string(args.slots_total) +
                                         " slots does not fit in shared memory with any CTA shape");
}

// Shared body of the evaluation entry points: validate and build, then launch.
fd_status eval_impl(const fd_graph *const *graphs, int32_t n_graphs, const fd_params *params,
                    const int32_t *graph_of_inst, int32_t n_inst, fd_vegas *const *maps,
                    const float *points, const float *point_w, uint64_t seed, uint64_t iter,
                    const uint32_t *iter_dev, int64_t n_per_inst, double *partials, float *per_sample_f,
                    int *status, cudaStream_t stream, float *abs_f = nullptr) {
    static thread_local EvalArgs args;   // large (kernel parameter space)
    const fd_status st = eval_build(graphs, n_graphs, params, graph_of_inst, n_inst, maps, points, point_w, seed,
                                    iter, iter_dev, n_per_inst, partials, per_sample_f, abs_f, status, args);
    if (st != FD_OK) return st;
    return eval_run(graphs, n_graphs, graph_of_inst, args, stream);
}
}  // namespace

extern "C" fd_status fd_debug_set_wait_polls(int64_t polls) {
    FD_REQUIRE(polls < (int64_t(1) << 32), "polls must be below 2^32");
    g_wait_polls.store(polls < 0 ? WAIT_LIMIT : (uint32_t)polls);
    return FD_OK;
}

extern "C" fd_status fd_integrand_eval(const fd_graph *const *graphs, int32_t n_graphs,
                                       const fd_params *params, const int32_t *graph_of_inst,
                                       int32_t n_inst, fd_vegas *const *maps, const float *points,
                                       const float *point_w, uint64_t seed, uint64_t iter,
                                       int64_t n_per_inst, double *partials, float *per_sample_f,
                                       void *stream) {
    return eval_impl(graphs, n_graphs, params, graph_of_inst, n_inst, maps, points, point_w, seed, iter, nullptr,
                     n_per_inst, partials, per_sample_f, fd::device_status_word(), (cudaStream_t)stream);
}

extern "C" fd_status fd_integrand_eval_target(const fd_graph *const *graphs, int32_t n_graphs,
                                              const fd_params *params, const int32_t *graph_of_inst,
                                              int32_t n_inst, fd_vegas *const *maps, const float *points,
                                              const float *point_w, uint64_t seed, uint64_t iter,
                                              int64_t n_per_inst, double *partials, float *abs_f,
                                              void *stream) {
    FD_REQUIRE(abs_f, "abs_f is required");
    return eval_impl(graphs, n_graphs, params, graph_of_inst, n_inst, maps, points, point_w, seed, iter, nullptr,
                     n_per_inst, partials, nullptr, fd::device_status_word(), (cudaStream_t)stream, abs_f);
}

extern "C" fd_status fd_integrand_eval_iter_dev(const fd_graph *const *graphs, int32_t n_graphs,
                                                const fd_params *params, const int32_t *graph_of_inst,
                                                int32_t n_inst, fd_vegas *const *maps, uint64_t seed,
                                                uint64_t iter_base, const uint32_t *d_iter, int64_t n_per_inst,
                                                double *partials, void *stream) {
    FD_REQUIRE(d_iter, "d_iter is required");
    return eval_impl(graphs, n_graphs, params, graph_of_inst, n_inst, maps, nullptr, nullptr, seed, iter_base,
                     d_iter, n_per_inst, partials, nullptr, fd::device_status_word(), (cudaStream_t)stream);
}

namespace {
__global__ void counter_add_kernel(uint32_t *c, uint32_t v) { *c += v; }
}  // namespace

extern "C" fd_status fd_counter_add(uint32_t *d_counter, uint32_t v, void *stream) {
    FD_REQUIRE(d_counter, "d_counter is required");
    counter_add_kernel<<<1, 1, 0, (cudaStream_t)stream>>>(d_counter, v);
    FD_CHECK_CUDA(cudaGetLastError());
    return FD_OK;
}

// ---- fd_accumulate ---------------------------------------------------------------
namespace {
// One warp per (instance, root, part): lane j sums tiles j, j + 32, ... with
// Neumaier compensation, then lane 0 combines the 32 lane sums in lane order
// (fixed order: bitwise reproducible).
__global__ void accumulate_kernel(const double *partials, int n_inst, int r_max, int tiles,
                                  int64_t n, double *out) {
    const int k = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);   // (inst, r, c)
    const int lane = threadIdx.x & 31;
    if (k >= n_inst * r_max * 2) return;
    const int inst = k / (r_max * 2), rc = k % (r_max * 2), r = rc / 2, c = rc % 2;
    double s = 0.0, sc = 0.0, q = 0.0, qc = 0.0;
    for (int t = lane; t < tiles; t += 32) {
        const double *p = partials + (((int64_t)inst * tiles + t) * r_max + r) * 4 + c * 2;
        neumaier(s, sc, p[0]);
        neumaier(q, qc, p[1]);
    }
    double ls[4] = {s, sc, q, qc};
    double S = 0.0, SC = 0.0, Q = 0.0, QC = 0.0;
    for (int j = 0; j < 32; ++j) {
        const double v0 = __shfl_sync(0xffffffffu, ls[0], j), v1 = __shfl_sync(0xffffffffu, ls[1], j);
        const double v2 = __shfl_sync(0xffffffffu, ls[2], j), v3 = __shfl_sync(0xffffffffu, ls[3], j);
        neumaier(S, SC, v0);
        neumaier(S, SC, v1);
        neumaier(Q, QC, v2);
        neumaier(Q, QC, v3);
    }
    if (lane != 0) return;
    S += SC;
    Q += QC;
    const double mean = S / (double)n;
    double var = 0.0;
    if (n > 1) var = fmax((Q - S * mean) / (double)(n - 1), 0.0) / (double)n;
    out[(((int64_t)inst * r_max + r) * 2 + c) * 2] = mean;
    out[(((int64_t)inst * r_max + r) * 2 + c) * 2 + 1] = var;
}
}  // namespace

extern "C" fd_status fd_accumulate(const double *partials, int32_t n_inst, int32_t r_max,
                                   int64_t n_per_inst, double *out, void *stream) {
    FD_REQUIRE(partials && out, "partials and out are required");
    FD_REQUIRE(n_inst > 0 && r_max > 0 && n_per_inst > 0, "sizes must be positive");
    const int64_t tl = fd_tile_samples(n_per_inst);
    const int tiles = (int)((n_per_inst + tl - 1) / tl);
    const int64_t threads = (int64_t)n_inst * r_max * 2 * 32;    // one warp per output
    accumulate_kernel<<<(unsigned)((threads + 127) / 128), 128, 0, (cudaStream_t)stream>>>(
        partials, n_inst, r_max, tiles, n_per_inst, out);
    FD_CHECK_CUDA(cudaGetLastError());
    return FD_OK;
}

// ---- the sampler map's cosine / sine table ---------------------------------------
// cos and sin of 2 pi n / 256, n = 0..256, each as a double-float pair (FP64
// libm values split into FP32 hi + lo), in every device's global memory; the
// double-float map (fd_sincos2pi_df) reads it.  Filled once per device, at
// the first graph load on that device (before any stream capture).
namespace {
__device__ __align__(16) FdTab4 g_sc_tab[257];
const FdTab4 *g_sc_tab_dev[64];
std::mutex g_sc_mu;
}  // namespace

namespace fd {
fd_status sc_table(const FdTab4 **out) {
    int dev = 0;
    FD_CHECK_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fd::set_error(FD_ENOTSUP, "device index beyond 63");
    std::lock_guard<std::mutex> lock(g_sc_mu);
    if (!g_sc_tab_dev[dev]) {
        FdTab4 h[257];
        for (int n = 0; n <= 256; ++n) {
            const double a = 2.0 * M_PI * (double)n / 256.0;
            const double c = std::cos(a), sn = std::sin(a);
            h[n].x = (float)c;
            h[n].y = (float)(c - (double)h[n].x);
            h[n].z = (float)sn;
            h[n].w = (float)(sn - (double)h[n].z);
        }
        FD_CHECK_CUDA(cudaMemcpyToSymbol(g_sc_tab, h, sizeof h));
        void *p = nullptr;
        FD_CHECK_CUDA(cudaGetSymbolAddress(&p, g_sc_tab));
        g_sc_tab_dev[dev] = static_cast<const FdTab4 *>(p);
    }
    *out = g_sc_tab_dev[dev];
    return FD_OK;
}
}  // namespace fd

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
    // every argument is checked before the shared array is written: a rejected
    // call leaves an earlier call's partial sums alone
    static thread_local EvalArgs args;
    st = eval_build(graphs, n_graphs, params, graph_of_inst, n_inst, maps, points, point_w, seed, iter, nullptr,
                    n_per_inst, partials, per_sample_f, nullptr, nullptr, args);
    if (st != FD_OK) return st;
    // every byte 0xFF is a NaN double: a tile the kernel failed to write shows up
    // as NaN in `out` instead of a stale value from an earlier call
    FD_CHECK_CUDA(cudaMemsetAsync(partials, 0xFF, (size_t)need * sizeof(double), s));
    st = eval_run(graphs, n_graphs, graph_of_inst, args, s);
    if (st != FD_OK) return st;
    return fd_accumulate(partials, n_inst, r_max, n_per_inst, out, stream);
}
